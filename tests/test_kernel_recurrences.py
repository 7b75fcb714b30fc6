"""The algebraic rewrites the CUDA inner iteration relies on, checked in FP64
numpy against the oracle's plain Hestenes-Stiefel CG (Sec. 2) on small dense
systems.  Each model below follows the kernels' order of operations:

  * V_hat^T p and V_hat^T s by recurrence instead of direct products, and the
    low-rank partial V_hat^T M_cg^{-1} q split as V_hat^T M_cg^{-1}(A p) + G c
    with G = V_hat^T M_cg^{-1} V_hat (two grid-wide reductions per iteration);
  * MINRES-CG* (Sec. 2.1, M_cg^{-1} = diag(A)^{-1} - 2 V_hat Lambda_hat^{-1}
    V_hat^T): V_hat^T r by recurrence and V_hat^T s = V_hat^T diag(A)^{-1} r +
    (V_hat^T V_hat) e with e = -2 Lambda_hat^{-1} V_hat^T r;
  * the one-kernel iteration (M_cg = I): each iteration updates r, then p,
    from the previous iteration's scalars, and the next residual norm comes
    from the expansion rho - 2 alpha r^T q + alpha^2 q^T q;
  * the one-gather iteration (M_cg = I or Jacobi): step a forms q = M_mr p
    with p explicit and, from the fresh rho_i = r_i^T s_i and the dots
    s^T q, q^T M_cg^{-1} q of the same iteration, beta_i by the expansion
    rho_i - 2 alpha s^T q + alpha^2 q^T M_cg^{-1} q; step b updates z, r and
    p = s + beta p and reduces the fresh rho_{i+1} for the next alpha;
  * the inner right-hand side normalised to unit length and the solution
    scaled back (CG is homogeneous).

Exact in exact arithmetic, so the models must reproduce the oracle's iterates
to rounding: a dropped term, a wrong sign or a stale value fails them."""
import numpy as np
import pytest

import oracle as O


def _csr(A):
    n = A.shape[0]
    rp, ci, va = [0], [], []
    for i in range(n):
        nz = np.nonzero(A[i])[0]
        ci += list(nz)
        va += list(A[i, nz])
        rp.append(len(ci))
    return np.array(rp, np.int64), np.array(ci, np.int32), np.array(va, np.float64)


def _system(n=40, k=3, seed=7):
    """Symmetric A with k negative eigenvalues, a positive diagonal that varies
    (so Jacobi and diag(A) differ from I) and a dense pattern."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    w = np.concatenate([-rng.uniform(0.1, 0.6, k), rng.uniform(0.4, 3.0, n - k)])
    S = np.diag(np.linspace(0.7, 1.4, n))
    A = S @ (Q * w) @ Q.T @ S
    A = (A + A.T) / 2
    ev, U = np.linalg.eigh(A)
    assert np.sum(ev < 0) == k and np.all(np.diag(A) > 0)
    V, lam = U[:, :k], ev[:k]
    return A, V, lam


def _ops(A, V, lam, mcg):
    c2 = 2.0 * np.abs(lam)
    if mcg == O.MCG_IDENTITY:
        minv = lambda r: r.copy()  # noqa: E731
    elif mcg == O.MCG_JACOBI:
        d = np.diag(A) + (V ** 2) @ c2
        minv = lambda r: r / d  # noqa: E731
    else:
        dA = np.diag(A)
        minv = lambda r: r / dA - V @ ((2.0 / lam) * (V.T @ r))  # noqa: E731
    return c2, minv


def _oracle_iterate(A, V, lam, y, m, mcg):
    s = O.System(*_csr(A), V, lam)
    z, it, st = s.cg(y, 1e-300, m, mcg)
    assert it == m and st == O.ERR_MAXITER
    return z


def _two_reduction_cg(A, V, lam, y, m, mcg):
    """Steps a and b of the inner iteration with the recurrences of the
    kernels; returns z_m and the largest gap between each recurred V_hat^T
    product and the direct one."""
    c2, minv = _ops(A, V, lam, mcg)
    G = V.T @ np.column_stack([minv(V[:, j]) for j in range(V.shape[1])])
    z = np.zeros_like(y)
    r = y.copy()
    s = minv(r)
    rho = r @ s
    vs = V.T @ s
    vp = np.zeros(V.shape[1])
    p = np.zeros_like(y)
    beta = 0.0
    gap = 0.0
    for _ in range(m):
        # step a: p' = s + beta p fused into the product, c from the recurred V^T p'
        p = s + beta * p
        vp = vs + beta * vp
        c = c2 * vp
        Ap = A @ p
        q = Ap + V @ c
        kappa = p @ q
        vq = V.T @ minv(Ap) + G @ c
        gap = max(gap, np.abs(vp - V.T @ p).max(), np.abs(vq - V.T @ minv(q)).max())
        # step b
        alpha = rho / kappa
        z = z + alpha * p
        r = r - alpha * q
        s = minv(r)
        rho_new = r @ s
        vs = vs - alpha * vq
        gap = max(gap, np.abs(vs - V.T @ s).max())
        beta = rho_new / rho
        rho = rho_new
    return z, gap


@pytest.mark.parametrize("mcg", [O.MCG_IDENTITY, O.MCG_JACOBI, O.MCG_SMW], ids=["identity", "jacobi", "smw"])
def test_recurred_low_rank_products_reproduce_cg(mcg):
    A, V, lam = _system()
    y = np.random.default_rng(3).standard_normal(A.shape[0])
    for m in (1, 2, 5, 12):
        z, gap = _two_reduction_cg(A, V, lam, y, m, mcg)
        zo = _oracle_iterate(A, V, lam, y, m, mcg)
        assert np.linalg.norm(z - zo) <= 1e-10 * np.linalg.norm(zo), m
        assert gap <= 1e-10 * np.linalg.norm(y)


def test_smw_projections_by_recurrence():
    """MINRES-CG*: V_hat^T r follows r's own recurrence and V_hat^T s is
    assembled from V_hat^T diag(A)^{-1} r and the Gram matrix V_hat^T V_hat."""
    A, V, lam = _system(seed=11)
    # columns scaled off unit length: the Gram term must be V^T V, not I
    V = V * (1.0 + 1e-3 * np.arange(V.shape[1]))
    _, minv = _ops(A, V, lam, O.MCG_SMW)
    dA = np.diag(A)
    VtV = V.T @ V
    rng = np.random.default_rng(5)
    r = rng.standard_normal(A.shape[0])
    vr = V.T @ r
    for _ in range(6):
        q = rng.standard_normal(A.shape[0])
        alpha = rng.uniform(0.1, 1.0)
        r = r - alpha * q
        vr = vr - alpha * (V.T @ q)
        e = -2.0 * vr / lam
        u = V.T @ (r / dA) + VtV @ e
        assert np.allclose(vr, V.T @ r, rtol=0, atol=1e-12 * np.linalg.norm(r))
        assert np.allclose(u, V.T @ minv(r), rtol=0, atol=1e-11 * np.linalg.norm(r))


def _one_kernel_cg(A, V, lam, y, m):
    """The one-kernel iteration (M_cg = I): iteration i first finishes
    iteration i-1's updates of its rows (r_i = r_{i-1} - alpha q_{i-1},
    p_i = r_i + beta p_{i-1}), then forms q_i = M_mr p_i and the dots
    r_i^T r_i, p_i^T q_i, r_i^T q_i, q_i^T q_i in one pass.  alpha_i uses the
    fresh rho_i; beta_i uses the expanded norm of r_{i+1}.  The last z update
    is applied after the loop.  Returns z_m and the expanded norms with the
    true ones."""
    c2, _ = _ops(A, V, lam, O.MCG_IDENTITY)
    M = lambda u: A @ u + V @ (c2 * (V.T @ u))  # noqa: E731
    z = np.zeros_like(y)
    r_prev = y.copy()
    q_prev = np.zeros_like(y)
    p = np.zeros_like(y)
    alpha = beta = 0.0
    pairs = []
    for i in range(m):
        r = r_prev - alpha * q_prev
        if i > 0:
            z = z + alpha * p
        p = r + beta * p
        q = M(p)
        rho, pq, rq, qq = r @ r, p @ q, r @ q, q @ q
        alpha = rho / pq
        rho_next = rho - 2.0 * alpha * rq + alpha * alpha * qq
        pairs.append((rho_next, np.linalg.norm(r - alpha * q) ** 2))
        beta = rho_next / rho
        r_prev, q_prev = r, q
    z = z + alpha * p  # the finishing kernel's pending update
    return z, pairs


def test_one_kernel_iteration_reproduces_cg():
    A, V, lam = _system(seed=13)
    y = np.random.default_rng(4).standard_normal(A.shape[0])
    for m in (1, 2, 6, 15):
        z, pairs = _one_kernel_cg(A, V, lam, y, m)
        zo = _oracle_iterate(A, V, lam, y, m, O.MCG_IDENTITY)
        assert np.linalg.norm(z - zo) <= 1e-10 * np.linalg.norm(zo), m
        for est, true in pairs:
            assert abs(est - true) <= 1e-10 * (y @ y)


def _one_gather_cg(A, V, lam, y, m, mcg):
    """Variants 9-11 with their step b: p is a stored vector (p_0 = s_0),
    step a reduces p^T q, s^T q, q^T M_cg^{-1} q and V^T M_cg^{-1} A p; its
    last block takes alpha from the fresh rho, beta from the expansion and
    advances V^T s, V^T p and c; step b applies z, r, p updates and reduces
    the fresh rho for the next iteration.  Returns z_m and the largest gaps of
    the expanded rho_{i+1} and of the recurred V^T p from the direct ones."""
    c2, minv = _ops(A, V, lam, mcg)
    dinv = minv(np.ones(A.shape[0]))  # the diagonal of M_cg^{-1} (identity or Jacobi)
    G = V.T @ (dinv[:, None] * V)
    z = np.zeros_like(y)
    r = y.copy()
    s = dinv * r
    p = s.copy()
    rho = r @ s
    vs = V.T @ s
    vp = vs.copy()
    gap_rho = gap_vp = 0.0
    for _ in range(m):
        # step a
        c = c2 * vp
        Ap = A @ p
        q = Ap + V @ c
        pq, sq, qdq = p @ q, s @ q, q @ (dinv * q)
        vq = V.T @ (dinv * Ap) + G @ c
        alpha = rho / pq
        rho_e = rho - 2.0 * alpha * sq + alpha * alpha * qdq
        beta = max(rho_e, 0.0) / rho
        vs = vs - alpha * vq
        vp = vs + beta * vp
        # step b
        z = z + alpha * p
        r = r - alpha * q
        s = dinv * r
        p = s + beta * p
        rho_fresh = r @ s
        gap_rho = max(gap_rho, abs(rho_e - rho_fresh))
        gap_vp = max(gap_vp, np.abs(vp - V.T @ p).max())
        rho = rho_fresh
    return z, gap_rho, gap_vp


@pytest.mark.parametrize("mcg", [O.MCG_IDENTITY, O.MCG_JACOBI], ids=["identity", "jacobi"])
def test_one_gather_iteration_reproduces_cg(mcg):
    A, V, lam = _system(seed=19)
    y = np.random.default_rng(8).standard_normal(A.shape[0])
    for m in (1, 2, 7, 16):
        z, gap_rho, gap_vp = _one_gather_cg(A, V, lam, y, m, mcg)
        zo = _oracle_iterate(A, V, lam, y, m, mcg)
        assert np.linalg.norm(z - zo) <= 1e-10 * np.linalg.norm(zo), m
        assert gap_rho <= 1e-10 * (y @ y) and gap_vp <= 1e-10 * np.linalg.norm(y)


def test_one_gather_model_detects_planted_mistakes():
    """The model fails when the expansion's cross term loses its factor 2 or
    beta comes from the previous iteration's rho: the pin is not vacuous."""
    A, V, lam = _system(seed=19)
    y = np.random.default_rng(8).standard_normal(A.shape[0])
    zo = _oracle_iterate(A, V, lam, y, 7, O.MCG_JACOBI)
    c2, minv = _ops(A, V, lam, O.MCG_JACOBI)
    dinv = minv(np.ones(A.shape[0]))
    M = lambda u: A @ u + V @ (c2 * (V.T @ u))  # noqa: E731
    for mistake in ("cross_term", "stale_beta"):
        z = np.zeros_like(y); r = y.copy(); s = dinv * r; p = s.copy(); rho = r @ s; rho_old = rho
        for _ in range(7):
            q = M(p)
            alpha = rho / (p @ q)
            cross = 1.0 if mistake == "cross_term" else 2.0
            rho_e = rho - cross * alpha * (s @ q) + alpha * alpha * (q @ (dinv * q))
            beta = rho_e / rho if mistake == "cross_term" else rho / rho_old
            z = z + alpha * p; r = r - alpha * q; s = dinv * r; p = s + beta * p
            rho_old, rho = rho, r @ s
        assert np.linalg.norm(z - zo) > 1e-6 * np.linalg.norm(zo), mistake


@pytest.mark.parametrize("mcg", [O.MCG_IDENTITY, O.MCG_JACOBI, O.MCG_SMW], ids=["identity", "jacobi", "smw"])
def test_inner_solve_of_the_normalised_rhs_scales_back(mcg):
    """The GPU solves M_mr z' = y/||y|| and returns ||y|| z': the same iterate
    and the same relative stopping test as CG on y."""
    A, V, lam = _system(seed=17)
    s = O.System(*_csr(A), V, lam)
    y = 1e3 * np.random.default_rng(6).standard_normal(A.shape[0])
    ny = np.linalg.norm(y)
    for m in (1, 4, 9):
        z1, it1, _ = s.cg(y, 1e-300, m, mcg)
        z2, it2, _ = s.cg(y / ny, 1e-300, m, mcg)
        assert it1 == it2 == m
        assert np.linalg.norm(ny * z2 - z1) <= 1e-12 * np.linalg.norm(z1)
    z1, it1, st1 = s.cg(y, 1e-6, 1000, mcg)
    z2, it2, st2 = s.cg(y / ny, 1e-6, 1000, mcg)
    assert it1 == it2 and st1 == st2 == O.OK
