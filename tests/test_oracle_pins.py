"""Pins for the FP64 CPU oracle: checks against mathematics the paper fixes.

Each test pins one oracle function to something other than itself: a closed
form, an identity from the paper, a textbook property of CG / MINRES, dense
numpy linear algebra, or hand-derived fixtures under tests/golden/.
"""
import os

import numpy as np
import pytest

import oracle as O
from gen import (batch64_lap2d, lap2d_64_k4, dense_to_csr, laplacian_csr, laplacian_smallest_eigs, random_sparse_symmetric,
                 random_indefinite_dense, shifted_family, shifted_laplacian_problem)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_system(n=40, k=3, seed=0):
    A, Vn, lam, d, Q = random_indefinite_dense(n, k, seed)
    rp, ci, va = dense_to_csr(A)
    return A, Vn, lam, d, Q, O.System(rp, ci, va, Vn, lam)


def dense_op(apply, n):
    return np.column_stack([apply(np.eye(n)[:, i]) for i in range(n)])


def absA(A):
    w, Q = np.linalg.eigh(A)
    return (Q * np.abs(w)) @ Q.T


# ---------------------------------------------------------------- M_mr (Sec. 2)

@pytest.mark.parametrize("k,seed", [(1, 1), (2, 2), (5, 3)])
def test_mmr_equals_abs_A_for_exact_subspace(k, seed):
    """Exact V_hat: M_mr = A + 2 V|L|V^T equals |A| = V|Lambda|V^T (Sec. 1-2)."""
    A, Vn, lam, d, Q, s = dense_system(40, k, seed)
    M = dense_op(s.mmr_apply, 40)
    assert np.allclose(M, absA(A), rtol=0, atol=1e-12 * np.abs(A).max())
    assert np.all(np.linalg.eigvalsh(0.5 * (M + M.T)) > 0)


def test_mmr_laplacian_spectrum_is_abs():
    """On a shifted 2D Laplacian with analytic eigenvectors, eig(M_mr) = |eig(A)|."""
    p = shifted_laplacian_problem("t", (7, 5), 3, seed=0)
    s = O.System.from_problem(p)
    M = dense_op(s.mmr_apply, p.n)
    wA = np.sort(np.abs(np.linalg.eigvalsh(p.dense())))
    wM = np.sort(np.linalg.eigvalsh(0.5 * (M + M.T)))
    assert np.allclose(wA, wM, atol=1e-12)


def test_mmr_smw_inverse():
    """Sec. 2.1: M_mr^{-1} = A^{-1} - 2 V Lambda^{-1} V^T, so M_mr applied to it is I."""
    A, Vn, lam, d, Q, s = dense_system(30, 4, 11)
    Minv = np.linalg.inv(A) - 2.0 * (Vn / lam) @ Vn.T
    rng = np.random.default_rng(0)
    for _ in range(3):
        u = rng.standard_normal(30)
        assert np.allclose(s.mmr_apply(Minv @ u), u, atol=1e-11)


def test_mmr_preconditioned_spectrum_pm1():
    """Sec. 1-2: eig(M_mr^{-1} A) are +1 and -1 only, with -1 of multiplicity k."""
    A, Vn, lam, d, Q, s = dense_system(36, 5, 5)
    M = dense_op(s.mmr_apply, 36)
    ev = np.linalg.eigvals(np.linalg.solve(M, A))
    assert np.allclose(np.abs(ev.imag), 0, atol=1e-9)
    ev = np.sort(ev.real)
    assert np.allclose(ev[:5], -1, atol=1e-9) and np.allclose(ev[5:], 1, atol=1e-9)


def test_mmr_flop_count():
    """Sec. 2: one M_mr product costs O(nnz + kn): exactly 2nnz + 4kn + k here."""
    p = shifted_laplacian_problem("t", (9, 8), 4, seed=1)
    s = O.System.from_problem(p)
    _, fl = s.mmr_apply(np.ones(p.n), count_flops=True)
    assert fl == 2 * p.nnz + 4 * p.k * p.n + p.k


def test_mmr_independent_of_basis_within_a_cluster():
    """M_mr depends on the negative invariant subspace, not on its basis
    (Sec. 2): rotating V_hat within a degenerate eigenvalue cluster and
    flipping column signs leaves every product unchanged, while mixing two
    columns of different eigenvalues changes it."""
    p = shifted_laplacian_problem("t", (9, 9), 3, seed=0)  # lambda_2 = lambda_3: modes (1,2), (2,1)
    assert p.k == 3 and p.lam[1] == p.lam[2] and p.lam[0] != p.lam[1]
    u = np.random.default_rng(8).standard_normal((p.n, 4))
    ref = O.System.from_problem(p)

    def mixed(i, j, t, flip):
        V = p.V.copy()
        c, sn = np.cos(t), np.sin(t)
        V[:, [i, j]] = p.V[:, [i, j]] @ np.array([[c, -sn], [sn, c]])
        V[:, flip] *= -1.0
        return O.System(p.rowptr, p.colind, p.val, V, p.lam)

    for t in (0.3, 1.1, 2.9):
        s = mixed(1, 2, t, 0)
        for col in u.T:
            y0 = ref.mmr_apply(col)
            assert np.linalg.norm(s.mmr_apply(col) - y0) <= 1e-13 * np.linalg.norm(y0)
    bad = mixed(0, 1, 0.3, 2)
    assert np.linalg.norm(bad.mmr_apply(u[:, 0]) - ref.mmr_apply(u[:, 0])) > 1e-3 * np.linalg.norm(u[:, 0])


def test_mmr_diag():
    A, Vn, lam, d, Q, s = dense_system(25, 3, 8)
    M = dense_op(s.mmr_apply, 25)
    assert np.allclose(s.mmr_diag(), np.diag(M), atol=1e-12)


def test_csr_spmv_matches_dense():
    p = shifted_laplacian_problem("t", (6, 5, 4), 2, seed=3)
    s = O.System.from_problem(p)
    x = np.random.default_rng(1).standard_normal(p.n)
    assert np.allclose(s.spmv(x), p.dense() @ x, rtol=0, atol=1e-13)


# ---------------------------------------------------------------- inner CG (Eq. 2)

def _krylov_galerkin(M, y, m, Dinv=None):
    """Textbook CG iterate: z_m in K_m(D^-1 M, D^-1 y) with M-orthogonal residual."""
    n = len(y)
    D = np.eye(n) if Dinv is None else np.diag(Dinv)
    vecs = [D @ y]
    for _ in range(m - 1):
        vecs.append(D @ (M @ vecs[-1]))
    K, _ = np.linalg.qr(np.column_stack(vecs))
    c = np.linalg.solve(K.T @ M @ K, K.T @ y)
    return K @ c


@pytest.mark.parametrize("mcg", [O.MCG_IDENTITY, O.MCG_JACOBI])
def test_cg_iterates_are_galerkin(mcg):
    """Each CG iterate is the energy-norm best approximation from the Krylov space (Sec. 2)."""
    A, Vn, lam, d, Q, s = dense_system(24, 2, 21)
    # make diag(M_mr) non-constant so Jacobi differs from identity
    Dsc = np.diag(np.linspace(0.5, 2.0, 24))
    A = Dsc @ A @ Dsc
    w, Qa = np.linalg.eigh(A)
    Vn, lam = Qa[:, :2], w[:2]
    assert np.all(lam < 0) and w[2] > 0
    rp, ci, va = dense_to_csr(A)
    s = O.System(rp, ci, va, Vn, lam)
    M = dense_op(s.mmr_apply, 24)
    y = np.random.default_rng(2).standard_normal(24)
    Dinv = 1.0 / np.diag(M) if mcg == O.MCG_JACOBI else None
    for m in range(1, 7):
        z, it, st = s.cg(y, 1e-300, m, mcg)
        assert it == m and st == O.ERR_MAXITER
        zg = _krylov_galerkin(M, y, m, Dinv)
        assert np.allclose(z, zg, rtol=0, atol=1e-9 * np.linalg.norm(zg))


def test_cg_energy_error_monotone_and_finite_termination():
    """Energy-norm error decreases monotonically (Sec. 2); exact after <= n steps."""
    rp, ci, va = laplacian_csr((4, 4))  # SPD, k = 0 so M_mr = A
    s = O.System(rp, ci, va)
    M = dense_op(s.mmr_apply, 16)
    y = np.random.default_rng(3).standard_normal(16)
    zs = np.linalg.solve(M, y)
    errs = []
    for m in range(1, 17):
        z, it, st = s.cg(y, 1e-300, m)
        e = z - zs
        errs.append(np.sqrt(e @ M @ e))
    assert all(b <= a * (1 + 1e-12) + 1e-14 for a, b in zip(errs, errs[1:]))
    z, it, st = s.cg(y, 1e-12, 16)
    assert st == O.OK and it <= 16
    assert np.linalg.norm(z - zs) <= 1e-10 * np.linalg.norm(zs)


def test_cg_stopping_rule():
    p = shifted_laplacian_problem("t", (10, 9), 3, seed=4)
    s = O.System.from_problem(p)
    y = np.random.default_rng(5).standard_normal(p.n)
    for tol in (1e-2, 1e-6):
        z, it, st = s.cg(y, tol, 10000)
        assert st == O.OK
        M = dense_op(s.mmr_apply, p.n)
        # recursive residual drift is tiny at this size: the true residual obeys the test
        assert np.linalg.norm(y - M @ z) <= tol * np.linalg.norm(y) * 1.01
        z1, it1, _ = s.cg(y, tol, it - 1)
        assert np.linalg.norm(y - M @ z1) > tol * np.linalg.norm(y)


def test_cg_indefinite_reports_not_spd():
    A = np.diag([-1.0, 1.0, 2.0, 3.0])
    rp, ci, va = dense_to_csr(A)
    s = O.System(rp, ci, va)  # k = 0: M_mr = A is indefinite
    z, it, st = s.cg(np.array([1.0, 0, 0, 0]), 1e-8, 10)
    assert st == O.ERR_NOT_SPD


def test_cg_zero_rhs():
    p = shifted_laplacian_problem("t", (5, 5), 1, seed=0)
    s = O.System.from_problem(p)
    z, it, st = s.cg(np.zeros(p.n), 1e-8, 10)
    assert st == O.OK and it == 0 and not z.any()


# ---------------------------------------------------------------- MINRES-CG* inner preconditioner (Sec. 2.1)

def test_smw_prec_is_exact_inverse_when_A_is_diagonal():
    """With A diagonal, Atilde = diag(A) = A is exact, so the Sec. 2.1 form
    diag(A)^{-1} - 2 V Lambda^{-1} V^T is M_mr^{-1} itself (= |A|^{-1}): it undoes
    M_mr, and the preconditioned CG converges in one iteration."""
    d = np.array([3.0, -0.5, 2.0, -4.0, 1.5, 0.25, -1.0, 5.0])
    neg = np.where(d < 0)[0]
    V = np.eye(len(d))[:, neg]
    rp, ci, va = dense_to_csr(np.diag(d))
    s = O.System(rp, ci, va, V, d[neg])
    u = np.random.default_rng(3).standard_normal(len(d))
    out, st = s.mcg_apply(s.mmr_apply(u), O.MCG_SMW)
    assert st == O.OK and np.allclose(out, u, rtol=0, atol=1e-14)
    z, it, st = s.cg(u, 1e-13, 10, O.MCG_SMW)
    assert st == O.OK and it == 1
    assert np.allclose(z, u / np.abs(d), rtol=0, atol=1e-14)


def test_smw_prec_spectrum_on_shifted_laplacian():
    """Exact V_hat and a constant diagonal c = 2d - sigma: on V the product
    M_cg^{-1} M_mr acts as (1/c - 2/lambda_j)|lambda_j| = |lambda_j|/c + 2, on the
    rest of the spectrum as lambda_i/c."""
    p = shifted_laplacian_problem("t", (7, 6), 4, seed=0)
    s = O.System.from_problem(p)
    M = dense_op(s.mmr_apply, p.n)
    P = dense_op(lambda r: s.mcg_apply(r, O.MCG_SMW)[0], p.n)
    c = 4.0 - p.sigma
    lamA = np.linalg.eigvalsh(p.dense())
    want = np.sort(np.concatenate([np.abs(lamA[:p.k]) / c + 2.0, lamA[p.k:] / c]))
    got = np.sort(np.linalg.eigvals(P @ M).real)
    assert np.allclose(got, want, rtol=0, atol=1e-11)


def test_smw_cg_iterates_are_galerkin():
    """With the Sec. 2.1 preconditioner P, each CG iterate is the M_mr-energy best
    approximation from K_m(P M_mr, P y)."""
    p = shifted_laplacian_problem("t", (6, 5), 3, seed=2)
    s = O.System.from_problem(p)
    M = dense_op(s.mmr_apply, p.n)
    P = dense_op(lambda r: s.mcg_apply(r, O.MCG_SMW)[0], p.n)
    y = np.random.default_rng(5).standard_normal(p.n)
    for m in range(1, 6):
        z, it, st = s.cg(y, 1e-300, m, O.MCG_SMW)
        assert it == m and st == O.ERR_MAXITER
        vecs = [P @ y]
        for _ in range(m - 1):
            vecs.append(P @ (M @ vecs[-1]))
        K, _ = np.linalg.qr(np.column_stack(vecs))
        zg = K @ np.linalg.solve(K.T @ M @ K, K.T @ y)
        assert np.allclose(z, zg, rtol=0, atol=1e-9 * np.linalg.norm(zg))


def test_smw_cuts_inner_iterations_when_negative_eigenvalues_are_small():
    """Sec. 2.1 / 4.3: the improvement pays off when the negative eigenvalues are
    the ones closest to zero.  With sigma near lambda_k the plain inner CG slows
    down while the MINRES-CG* inner CG does not."""
    y = None
    counts = {}
    for frac in (0.5, 0.02):
        p = shifted_laplacian_problem("t", (24, 20), 4, seed=0, sigma_frac=frac)
        s = O.System.from_problem(p)
        y = np.random.default_rng(0).standard_normal(p.n)
        counts[frac] = [s.cg(y, 1e-6, 100000, mcg)[1] for mcg in (O.MCG_IDENTITY, O.MCG_SMW)]
    assert counts[0.5][1] < counts[0.5][0]
    assert counts[0.02][0] > 1.2 * counts[0.5][0]        # plain CG slows down
    assert counts[0.02][1] <= counts[0.5][1] + 2          # MINRES-CG* does not
    assert counts[0.02][1] < 0.7 * counts[0.02][0]


def test_smw_rejects_zero_diagonal():
    """A saddle-point row with a zero diagonal leaves diag(A) singular."""
    A = np.array([[2.0, 1.0], [1.0, 0.0]])
    rp, ci, va = dense_to_csr(A)
    s = O.System(rp, ci, va)
    out, st = s.mcg_apply(np.ones(2), O.MCG_SMW)
    assert st == O.ERR_INVALID
    z, it, st = s.cg(np.ones(2), 1e-8, 10, O.MCG_SMW)
    assert st == O.ERR_INVALID


def test_minres_cg_star_dense_solution():
    """MINRES-CG* (Alg. 1 with the Sec. 2.1 inner preconditioner) solves A x = b."""
    p = shifted_laplacian_problem("t", (9, 8), 4, seed=6, sigma_frac=0.1)
    r = O.minres_cg(O.System.from_problem(p), p.b, outer_tol=1e-12, inner_tol=1e-3, mcg=O.MCG_SMW)
    assert r.status == O.OK
    assert np.allclose(r.x, np.linalg.solve(p.dense(), p.b), rtol=0, atol=1e-8 * np.abs(p.xstar).max() * 10)


# ---------------------------------------------------------------- outer MINRES

def test_minres_identity_prec_matches_residual_norm():
    """P = I: MINRES minimises ||r||_2, so |eta_j| = ||b - A x_j|| and is monotone."""
    A, Vn, lam, d, Q, s = dense_system(30, 4, 13)
    b = np.random.default_rng(4).standard_normal(30)
    r = O.minres(s, b, lambda v: v, outer_tol=1e-13, restart_factor=0.0)  # no restarts
    assert r.status == O.OK and r.restarts == 0
    bn = np.linalg.norm(b)
    assert np.allclose(r.eta_history / bn, r.relres_history, rtol=1e-6, atol=1e-14)
    assert np.all(np.diff(r.eta_history) <= 1e-14)
    assert np.allclose(r.x, np.linalg.solve(A, b), atol=1e-10)
    assert r.outer_iters <= 30 + 2


def test_minres_spd_prec_minimises_prec_norm():
    """SPD P: |eta_j| = ||r_j||_{P^{-1}}, and it is non-increasing."""
    A, Vn, lam, d, Q, s = dense_system(20, 3, 17)
    rng = np.random.default_rng(6)
    G = rng.standard_normal((20, 20))
    P = G @ G.T + 20 * np.eye(20)
    b = rng.standard_normal(20)
    Pinv = np.linalg.inv(P)
    etas = []
    for j in range(1, 9):
        r = O.minres(s, b, lambda v: np.linalg.solve(P, v), outer_tol=1e-300, max_outer=j, restart_factor=0.0)
        assert r.outer_iters == j
        res = b - A @ r.x
        etas.append(r.eta_history[-1])
        assert np.isclose(r.eta_history[-1], np.sqrt(res @ Pinv @ res), rtol=1e-8)
    assert all(b <= a * (1 + 1e-12) for a, b in zip(etas, etas[1:]))


def test_minres_exact_mmr_converges_in_two_steps():
    """Sec. 1-2: with the exact M_mr, M_mr^{-1}A has eigenvalues +-1: <= 2 iterations."""
    A, Vn, lam, d, Q, s = dense_system(50, 6, 23)
    M = dense_op(s.mmr_apply, 50)
    L = np.linalg.cholesky(0.5 * (M + M.T))
    prec = lambda v: np.linalg.solve(L.T, np.linalg.solve(L, v))
    b = np.random.default_rng(7).standard_normal(50)
    r = O.minres(s, b, prec, outer_tol=1e-12, restart_factor=0.0)
    assert r.status == O.OK and r.outer_iters <= 2
    assert np.allclose(r.x, np.linalg.solve(A, b), atol=1e-10)


def _min_residual_iterate(A, b, xc, j):
    """x in xc + K_j(A, b - A xc) of least 2-norm residual: an orthonormal basis
    of the Krylov space (Gram-Schmidt, twice) and a dense least-squares solve.
    This is the defining property of MINRES with P = I, computed without its
    Lanczos / Givens recurrences."""
    r0 = b - A @ xc
    Q = np.zeros((len(b), j))
    q = r0 / np.linalg.norm(r0)
    for i in range(j):
        for _ in range(2):
            q = q - Q[:, :i] @ (Q[:, :i].T @ q)
        Q[:, i] = q / np.linalg.norm(q)
        q = A @ Q[:, i]
    y, *_ = np.linalg.lstsq(A @ Q, r0, rcond=None)
    return xc + Q @ y


def _restarted_minres_model(A, b, f, steps, window=3, restart_from_current=True):
    """Restarted MINRES (P = I) by the reading of the restart rule: within a
    cycle, after its j-th step (j > window), restart when
    relres_j > f * relres_{j - window}; the next cycle's Krylov space is built
    on b - A x at the current x.  Returns (x, relres history, restart steps,
    smallest |log(ratio / f)| over the decisions taken)."""
    bn = np.linalg.norm(b)
    xc = np.zeros(len(b))
    cyc, hist, restarts, margin = [], [], [], np.inf
    x = xc
    for step in range(1, steps + 1):
        x = _min_residual_iterate(A, b, xc, len(cyc) + 1)
        rr = np.linalg.norm(b - A @ x) / bn
        hist.append(rr)
        cyc.append(rr)
        m = len(cyc)
        if m > window:
            ratio = rr / cyc[m - 1 - window]
            margin = min(margin, abs(np.log(ratio / f)))
            if ratio > f:
                restarts.append(step)
                xc = x.copy() if restart_from_current else np.zeros(len(b))
                cyc = []
    return x, np.array(hist), restarts, margin


def test_minres_restart_rule_matches_restarted_least_squares_model():
    """Restart safeguard (the paper is silent; the reading: restart a cycle from
    the current x when relres_j > f * relres_{j-3}, j >= 4 within the cycle).
    With P = I every MINRES iterate is the least-residual point of its cycle's
    Krylov space, so a dense least-squares model of restarted MINRES fixes the
    whole residual history, the steps at which cycles restart and the final x.
    The decisions are taken with a margin of at least 10 % from f, and the model
    restarts at steps 5, 9 and 13 (a first cycle of five steps, then cycles of
    four), so a shifted window or a cycle restarted from the wrong point gives a
    different history."""
    rng = np.random.default_rng(7)
    n = 40
    lam = np.concatenate([-rng.uniform(0.05, 1.0, 6), rng.uniform(0.05, 1.0, n - 6)])
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (Qm * lam) @ Qm.T
    A = 0.5 * (A + A.T)
    b = rng.standard_normal(n)
    rp, ci, va = dense_to_csr(A)
    s = O.System(rp, ci, va)
    f, steps = 0.6, 14
    x, hist, restarts, margin = _restarted_minres_model(A, b, f, steps)
    assert restarts == [5, 9, 13] and margin > 0.1
    r = O.minres(s, b, lambda v: v, outer_tol=1e-300, max_outer=steps, restart_factor=f)
    assert r.outer_iters == steps and r.restarts == len(restarts)
    assert np.allclose(r.relres_history, hist, rtol=1e-10, atol=0)
    assert np.linalg.norm(r.x - x) <= 1e-10 * np.linalg.norm(x)
    # the model is sensitive to the two mistakes the pin is for
    _, h_shift, rs_shift, _ = _restarted_minres_model(A, b, f, steps, window=2)
    _, h_zero, _, _ = _restarted_minres_model(A, b, f, steps, restart_from_current=False)
    assert rs_shift != restarts or not np.allclose(h_shift, hist, rtol=1e-6)
    assert not np.allclose(h_zero, hist, rtol=1e-6)
    # f < 0 turns the rule off: no restart, and the history is monotone (P = I)
    r0 = O.minres(s, b, lambda v: v, outer_tol=1e-300, max_outer=steps, restart_factor=-1.0)
    assert r0.restarts == 0 and np.all(np.diff(r0.relres_history) <= 1e-14)


def test_minres_cg_dense_solution():
    """Alg. 1 end to end on a tiny dense problem: x equals the LU solution."""
    A, Vn, lam, d, Q, s = dense_system(60, 5, 29)
    b = np.random.default_rng(8).standard_normal(60)
    r = O.minres_cg(s, b, outer_tol=1e-13, inner_tol=1e-3)
    assert r.status == O.OK
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(r.x - xs) <= 1e-10 * np.linalg.norm(xs)
    assert r.true_relres <= 1e-13
    assert np.isclose(r.true_relres, np.linalg.norm(b - A @ r.x) / np.linalg.norm(b), rtol=1e-6)


def test_minres_cg_lap2d_64_matches_xstar():
    """64x64 shifted Laplacian (4 negatives): x* is recovered to kappa * tol."""
    p = lap2d_64_k4()
    s = O.System.from_problem(p)
    r = O.minres_cg(s, p.b, outer_tol=1e-12, inner_tol=1e-3)
    assert r.status == O.OK and r.true_relres <= 1e-12
    err = np.linalg.norm(r.x - p.xstar) / np.linalg.norm(p.xstar)
    assert err <= 1e-8
    assert np.isclose(s.true_relres(p.b, r.x), r.true_relres, rtol=1e-9)
    assert r.inner_iters_total > 0 and r.prec_calls == r.outer_iters + 1 + r.restarts


def test_minres_cg_jacobi_and_k0():
    p = shifted_laplacian_problem("t", (9, 7), 3, seed=9)
    s = O.System.from_problem(p)
    r = O.minres_cg(s, p.b, outer_tol=1e-12, inner_tol=1e-3, mcg=O.MCG_JACOBI)
    assert r.status == O.OK and np.allclose(r.x, p.xstar, atol=1e-8)
    rp, ci, va = laplacian_csr((9, 7))  # SPD, no negative eigenvalues: M_mr = A
    s0 = O.System(rp, ci, va)
    b = np.random.default_rng(3).standard_normal(63)
    r0 = O.minres_cg(s0, b, outer_tol=1e-12, inner_tol=1e-3)
    assert r0.status == O.OK
    assert np.allclose(r0.x, np.linalg.solve(s0_dense(rp, ci, va, 63), b), atol=1e-9)


def s0_dense(rp, ci, va, n):
    import scipy.sparse as sp
    return sp.csr_matrix((va, ci, rp), shape=(n, n)).toarray()


def test_minres_cg_degenerate_inputs():
    p = shifted_laplacian_problem("t", (8, 8), 4, seed=2)
    s = O.System.from_problem(p)
    r = O.minres_cg(s, np.zeros(p.n))
    assert r.status == O.OK and not r.x.any() and r.outer_iters == 0
    r = O.minres_cg(s, p.b, x0=p.xstar, outer_tol=1e-10)
    assert r.status == O.OK and r.outer_iters == 0
    r = O.minres_cg(s, p.b, outer_tol=1e-12, max_iters=5)
    assert r.status == O.ERR_MAXITER and r.inner_iters_total <= 5
    b = p.b.copy(); b[3] = np.nan
    assert O.minres_cg(s, b).status == O.ERR_NONFINITE


def test_inexact_preconditioned_spectrum_clusters():
    """Sec. 4.2 (eigenvalue figures): P_inexact A clusters at +-1 and tightens with the inner tolerance."""
    A, Vn, lam, d, Q, s = dense_system(40, 3, 31)
    dist = []
    for tol in (1e-2, 1e-4, 1e-6):
        T = np.column_stack([s.cg(A[:, i], tol, 10000)[0] for i in range(40)])
        ev = np.linalg.eigvals(T)
        dd = np.minimum(np.abs(ev - 1), np.abs(ev + 1))
        dist.append(dd.max())
        assert np.sum(ev.real < 0) == 3
    assert dist[0] > dist[1] > dist[2] and dist[2] < 1e-3


# ---------------------------------------------------------------- 2x2 replacement (Sec. 1)

def _golden_2x2():
    rows = []
    with open(os.path.join(GOLDEN, "abs_2x2.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                a, e, o = (np.array(part.split(), dtype=float) for part in line.split("|"))
                rows.append((a, e, o))
    return rows


@pytest.mark.parametrize("case", _golden_2x2())
def test_abs_2x2_golden(case):
    (a, b, c), eig, out = case
    B, (l1, l2), (cs, sn) = O.abs_2x2(a, b, c)
    assert np.allclose(sorted([l1, l2]), sorted(eig), atol=1e-14)
    assert np.allclose(B, [[out[0], out[1]], [out[1], out[2]]], atol=1e-14)


def test_abs_2x2_closed_form_and_reflector():
    rng = np.random.default_rng(9)
    for _ in range(200):
        a, b, c = rng.standard_normal(3) * rng.choice([1e-3, 1, 1e3])
        Bt, (l1, l2), (cs, sn) = O.abs_2x2(a, b, c)
        B = np.array([[a, b], [b, c]])
        R = np.array([[cs, sn], [sn, -cs]])
        assert np.isclose(cs * cs + sn * sn, 1.0)
        assert np.allclose(R @ np.diag([l1, l2]) @ R, B, atol=1e-12 * np.abs(B).max())
        closed = (B @ B + abs(np.linalg.det(B)) * np.eye(2)) / (abs(l1) + abs(l2))
        assert np.allclose(Bt, closed, atol=1e-12 * np.abs(B).max())
        # n = 2 case of the deflation: B + 2 |l_-| v_- v_-^T
        w, Q = np.linalg.eigh(B)
        D = B.copy()
        for i in range(2):
            if w[i] < 0:
                D += 2 * abs(w[i]) * np.outer(Q[:, i], Q[:, i])
        assert np.allclose(Bt, D, atol=1e-12 * np.abs(B).max())


# ---------------------------------------------------------------- generators

@pytest.mark.parametrize("dims,k", [((64, 64), 4), ((7, 5), 3), ((6, 5, 4), 2), ((5, 5, 5), 2), ((8, 8), 2)])
def test_generator_inertia_and_eigenpairs(dims, k):
    """Negative count equals k (raised past ties); V, Lambda are eigenpairs of A."""
    p = shifted_laplacian_problem("t", dims, k, seed=0)
    A = p.dense()
    w = np.linalg.eigvalsh(A)
    assert int(np.sum(w < 0)) == p.k >= k
    assert np.allclose(np.sort(p.lam), w[: p.k], atol=1e-12)
    assert np.abs(A @ p.V - p.V * p.lam).max() <= 1e-12
    assert np.abs(p.V.T @ p.V - np.eye(p.k)).max() <= 1e-12
    assert np.allclose(A @ p.xstar, p.b, atol=1e-13)


def test_generator_tie_rounding():
    # cube: eigenvalues come in clusters (2,1,1)x3 etc.: k = 2 must round up to 4
    p = shifted_laplacian_problem("t", (5, 5, 5), 2, seed=0)
    assert p.k == 4
    ev = laplacian_smallest_eigs((64, 64), 6)
    assert np.isclose(ev[0][0], 2 * (2 - 2 * np.cos(np.pi / 65)))
    assert np.isclose(p.sigma, 0.5 * (laplacian_smallest_eigs((5, 5, 5), 5)[3][0] +
                                      laplacian_smallest_eigs((5, 5, 5), 5)[4][0]))


def test_shifted_family_columns_are_the_stated_systems():
    """Every column c = j * nrhs + r of a shifted family is (L - sigma_j I) x = b
    with exactly k_j negative eigenvalues (dense eigvalsh), sigma_j midway
    between eigenvalues k_j and k_j + 1 of L, V_hat_j / Lambda_hat_j its
    negative eigenpairs, and b = A x*."""
    fam = shifted_family((6, 5, 4), 3, 2, 8, seed=9)
    rp, ci, va = laplacian_csr((6, 5, 4))
    L = np.zeros((fam.n, fam.n))
    for i in range(fam.n):
        L[i, ci[rp[i]:rp[i + 1]]] = va[rp[i]:rp[i + 1]]
    wL = np.linalg.eigvalsh(L)
    assert np.allclose(fam.lamL, wL[:len(fam.lamL)], atol=1e-12)
    assert fam.ncols == 6 and fam.B.shape == (fam.n, 6)
    for c in range(fam.ncols):
        j = c // fam.nrhs
        p = fam.column_problem(c)
        A = p.dense()
        assert np.allclose(A, L - fam.sigma[j] * np.eye(fam.n), atol=0)
        w = np.linalg.eigvalsh(A)
        kj = int(fam.k[j])
        assert p.k == kj and int(np.sum(w < 0)) == kj
        assert np.isclose(fam.sigma[j], 0.5 * (wL[kj - 1] + wL[kj]), rtol=0, atol=1e-12)
        assert np.abs(A @ p.V - p.V * p.lam).max() <= 1e-12
        assert np.allclose(A @ fam.xstar[:, c], fam.B[:, c], atol=1e-13)


def test_batch_generator_draws_squares_and_rounded_k():
    """Uneven batch: square sides in the stated range, k_i raised to the end of
    its cluster (exactly k_i negative analytic eigenvalues), one RHS each."""
    ps = batch64_lap2d(count=6, sides=(8, 14), kmax=6, seed=3)
    for p in ps:
        m_ = int(round(np.sqrt(p.n)))
        assert m_ * m_ == p.n and 8 <= m_ <= 14
        w = np.linalg.eigvalsh(p.dense())
        assert int(np.sum(w < 0)) == p.k and 1 <= p.k
        assert p.xstar is None and p.b.shape == (p.n,) and np.all(np.abs(p.b) <= 1.0)


def test_generator_is_reproducible():
    a, b = lap2d_64_k4(), lap2d_64_k4()
    assert np.array_equal(a.b, b.b) and np.array_equal(a.V, b.V) and a.sigma == b.sigma


# ---------------------------------------------------------------- saddle-point generator

def test_saddle_inertia_and_eigenpairs():
    """[K B^T; B 0] with K SPD, B full row rank: exactly nb negative eigenvalues (Sylvester)."""
    from gen import small_saddle
    p = small_saddle()
    w = np.linalg.eigvalsh(p.dense())
    assert int(np.sum(w < 0)) == p.k == 6
    assert np.allclose(np.sort(p.lam), w[:6], atol=1e-12)
    assert p.meta["eig_residual_max"] < 1e-11
    s = O.System.from_problem(p)
    r = O.minres_cg(s, p.b, outer_tol=1e-12, inner_tol=1e-3)
    assert r.status == O.OK
    assert np.linalg.norm(r.x - p.xstar) <= 1e-8 * np.linalg.norm(p.xstar)


def test_saddle_krylov_eigensolver_matches_dense():
    """The Rayleigh-Ritz eigensolver of the large saddle generator agrees with dense eigh."""
    torch = pytest.importorskip("torch")
    from gen.saddle import _negative_eigenpairs_dense, _negative_eigenpairs_krylov, saddle_matrix
    A, K, B, _ = saddle_matrix(10, 8, 16, 4)
    Vk, lk = _negative_eigenpairs_krylov(K, B, 8, -0.3, 12, device="cpu")
    Vd, ld = _negative_eigenpairs_dense(A, 8)
    assert np.allclose(lk, ld, atol=1e-12)
    assert np.linalg.norm(A @ Vk - Vk * lk, axis=0).max() < 1e-10
    assert np.linalg.svd(Vk.T @ Vd, compute_uv=False).min() > 1 - 1e-10



# ---------------------------------------------------------------- setup stage 2: negative eigenpairs

def test_dense_negative_eigenpairs_match_laplacian_spectrum_and_inertia():
    """The dense stage-2 reference returns the analytic negative spectrum of a
    shifted Laplacian (sine-mode eigenvalues) with an orthonormal basis of
    A-invariant vectors, and Sylvester's count on a saddle system."""
    p = shifted_laplacian_problem("eig_pin", (13, 11), 5, seed=3)
    V, lam, w = O.negative_eigenpairs_dense(p.rowptr, p.colind, p.val)
    assert len(lam) == p.k
    assert np.allclose(lam, p.lam, rtol=0, atol=1e-12)
    A = p.dense()
    assert np.allclose(A @ V, V * lam, atol=1e-11)
    assert np.allclose(V.T @ V, np.eye(p.k), atol=1e-12)
    from gen import small_saddle
    q = small_saddle()
    V2, lam2, _ = O.negative_eigenpairs_dense(q.rowptr, q.colind, q.val)
    assert len(lam2) == q.k  # nb constraint rows: Sylvester's law of inertia


# ---------------------------------------------------------------- ILU(0) inner preconditioner (Sec. 4)

def _dense(rp, ci, va):
    n = len(rp) - 1
    A = np.zeros((n, n))
    for i in range(n):
        A[i, ci[rp[i]:rp[i + 1]]] = va[rp[i]:rp[i + 1]]
    return A


def test_ilu0_of_a_tridiagonal_matrix_is_its_exact_lu():
    """Tridiagonal A (indefinite, nonzero pivots): ILU(0) has no fill to drop,
    so L U = A and the preconditioner is A^{-1}."""
    rp, ci, va = laplacian_csr((31,), sigma=0.37)
    A = _dense(rp, ci, va)
    s = O.System(rp, ci, va)
    assert s.set_ilu0() == O.OK
    L, U = s.ilu0_factors()
    assert np.allclose(L @ U, A, atol=1e-13)
    r = np.random.default_rng(1).standard_normal(31)
    assert np.allclose(s.ilu0_apply(r), np.linalg.solve(A, r), atol=1e-10)


def test_ilu0_matches_a_on_its_pattern_and_solves_triangularly():
    """General sparse pattern: L is unit lower and U upper triangular on A's
    pattern, (L U)_ij = a_ij wherever a_ij is stored (the defining property of
    ILU(0)), fill outside the pattern is dropped, and the preconditioner is the
    two triangular solves (scipy's solve_triangular)."""
    from scipy.linalg import solve_triangular
    rp, ci, va = random_sparse_symmetric(60, 5, density_rows=(2, 9), diag_shift=6.0, empty_rows=0)
    A = _dense(rp, ci, va)
    pattern = A != 0
    s = O.System(rp, ci, va)
    assert s.set_ilu0() == O.OK
    L, U = s.ilu0_factors()
    assert np.allclose(np.diag(L), 1.0) and np.allclose(np.triu(L, 1), 0) and np.allclose(np.tril(U, -1), 0)
    assert not np.any((L - np.eye(60) != 0) & ~pattern) and not np.any((U != 0) & ~pattern)
    LU = L @ U
    assert np.allclose(LU[pattern], A[pattern], atol=1e-12)
    assert np.abs(LU[~pattern]).max() > 1e-3  # fill was dropped, so L U is not A
    r = np.random.default_rng(2).standard_normal(60)
    ref = solve_triangular(U, solve_triangular(L, r, lower=True, unit_diagonal=True), lower=False)
    assert np.allclose(s.ilu0_apply(r), ref, atol=1e-12)


def test_block_jacobi_ilu0_factors_each_diagonal_block():
    """Blocks of b rows: M = L U is block diagonal, and each block is the
    ILU(0) of A's diagonal block factored on its own (couplings between
    blocks dropped)."""
    rp, ci, va = laplacian_csr((7, 6), sigma=0.5)
    A = _dense(rp, ci, va)
    n, b = 42, 8
    s = O.System(rp, ci, va)
    assert s.set_ilu0(b) == O.OK
    L, U = s.ilu0_factors()
    M = L @ U
    for i0 in range(0, n, b):
        i1 = min(i0 + b, n)
        Ab = A[i0:i1, i0:i1]
        sb = O.System(*dense_to_csr(Ab))
        assert sb.set_ilu0() == O.OK
        Lb, Ub = sb.ilu0_factors()
        assert np.allclose(M[i0:i1, i0:i1], Lb @ Ub, atol=1e-13)
        M[i0:i1, i0:i1] = 0.0
    assert np.allclose(M, 0.0)


def test_ilu0_zero_pivot_is_a_breakdown():
    A = np.array([[0.0, 1.0], [1.0, 2.0]])
    s = O.System(*dense_to_csr(A))
    assert s.set_ilu0() == O.ERR_BREAKDOWN


@pytest.mark.parametrize("mcg", [O.MCG_ILU0, O.MCG_SMW_ILU0], ids=["ilu0", "smw_ilu0"])
def test_ilu_cg_iterates_are_galerkin(mcg):
    """CG on M_mr with P = M_cg^{-1} (ILU(0), or the MINRES-CG* form with
    Atilde = ILU(0)): iterates are the M_mr-energy best points of
    K_m(P M_mr, P y) -- P is symmetric here because A is (U = D L^T)."""
    A, Vn, lam, d, Q, s0 = dense_system(30, 3, 31)
    A = A + 0.0  # dense symmetric, every pivot nonzero for this seed
    rp, ci, va = dense_to_csr(A)
    s = O.System(rp, ci, va, Vn, lam)
    assert s.set_ilu0() == O.OK
    M = dense_op(s.mmr_apply, 30)
    P = dense_op(lambda r: s.mcg_apply(r, mcg)[0], 30)
    assert np.allclose(P, P.T, atol=1e-9 * np.abs(P).max())
    y = np.random.default_rng(3).standard_normal(30)
    for m_it in range(1, 6):
        z, it, st = s.cg(y, 1e-300, m_it, mcg)
        assert it == m_it
        vecs = [P @ y]
        for _ in range(m_it - 1):
            vecs.append(P @ (M @ vecs[-1]))
        K, _ = np.linalg.qr(np.column_stack(vecs))
        zg = K @ np.linalg.solve(K.T @ M @ K, K.T @ y)
        assert np.allclose(z, zg, rtol=0, atol=1e-8 * np.linalg.norm(zg))


def test_ilu0_cuts_inner_iterations_on_a_laplacian():
    """On a shifted 2D Laplacian the ILU(0) inner preconditioner (one block)
    needs fewer CG iterations than M_cg = I to the same tolerance, and
    MINRES-CG with it reaches x*."""
    p = shifted_laplacian_problem("ilu_lap", (30, 29), 5, seed=7)
    s = O.System.from_problem(p)
    assert s.set_ilu0() == O.OK
    y = np.random.default_rng(4).standard_normal(p.n)
    _, it_id, st_id = s.cg(y, 1e-6, 10000, O.MCG_IDENTITY)
    _, it_ilu, st_ilu = s.cg(y, 1e-6, 10000, O.MCG_ILU0)
    assert st_id == st_ilu == O.OK and it_ilu < it_id
    r = O.minres_cg(s, p.b, outer_tol=1e-12, inner_tol=1e-3, mcg=O.MCG_ILU0)
    assert r.status == O.OK
    assert np.linalg.norm(r.x - p.xstar) / np.linalg.norm(p.xstar) <= 1e-8
