"""Pins for the dense reference of the complex shifted systems (Sec. 3).

The section's algebra is checked on a small synthetic disk-brake stand-in:
the real-equivalent system reproduces the complex solution; the block LU of
the preconditioner M is exact; the Schur complement factors as S = S1 S2;
S2t is S2 without its (1, 2) block and its diagonal block is
-(1/gamma_i)(KE - |gamma|^2 Mass), whose inertia is the generator's k; the
block-LU application equals M^{-1} r; and S2t preconditions S2 well inside
GMRES, while the plain splitting iteration with S2t diverges.
"""
import numpy as np

from gen import small_brake
from oracle import complex_shifted as CS


def _sys():
    s = small_brake()
    return s, s.KE.toarray(), s.K.toarray(), s.D.toarray()


def test_real_equivalent_system_reproduces_the_complex_solution():
    s, KE, K, D = _sys()
    x, y = CS.complex_solve(K, D, s.mass, s.gamma, s.f, s.g)
    R = CS.real_equivalent(K, D, s.mass, s.gamma)
    z = np.linalg.solve(R, np.concatenate([s.g, s.f]))
    n2 = 2 * s.n
    assert np.allclose(z[:n2], x, atol=1e-10 * np.abs(x).max())
    assert np.allclose(z[n2:], -y, atol=1e-10 * np.abs(y).max())
    A, B = CS.companion(K, D, s.mass)
    C = s.gamma * B - A
    assert np.allclose(C @ (x + 1j * y), s.f + 1j * s.g, atol=1e-9)


def test_preconditioner_block_lu_and_schur_factorisation():
    s, KE, K, D = _sys()
    At, Bt, S, S1, S2, S2t, Di = CS.precond_blocks(KE, s.mass, s.gamma)
    n2 = 2 * s.n
    M = np.block([[Bt, -At], [At, Bt]])
    Lf = np.block([[Bt, np.zeros((n2, n2))], [At, S]])
    Uf = np.block([[np.eye(n2), -np.linalg.solve(Bt, At)], [np.zeros((n2, n2)), np.eye(n2)]])
    assert np.allclose(Lf @ Uf, M, atol=1e-9 * np.abs(M).max())
    assert np.allclose(S1 @ S2, S, atol=1e-9 * np.abs(S).max())
    n = s.n
    assert np.allclose(S2t[:n, n:], 0.0) and np.allclose(S2t[:n, :n], S2[:n, :n])
    assert np.allclose(S2t[n:, :], S2[n:, :])
    g = s.gamma
    assert np.allclose(Di, -(KE - abs(g) ** 2 * np.diag(s.mass)) / g.imag)
    # the inner level has the generator's k negative eigenvalues
    w = np.linalg.eigvalsh(CS.inner_level_matrix(KE, s.mass, s.gamma))
    assert np.sum(w < 0) == s.k
    assert np.allclose(np.sort(w[: s.k]), np.sort(s.lam), atol=1e-10)


def test_precond_apply_is_the_inverse_of_M_and_S2t_preconditions_S2():
    """The block-LU application equals M^-1 r; and S2t is a good preconditioner
    for S2 in a Krylov method (Sec. 3): GMRES on S2 with S2t^-1 as right
    preconditioner (scipy) reaches 1e-10 in few iterations, although S2t is
    not close enough to S2 for a plain splitting iteration (the inner-level
    matrix has eigenvalues near zero, so S2t^-1 is large on those modes)."""
    import scipy.sparse.linalg as spla
    s, KE, K, D = _sys()
    At, Bt, S, S1, S2, S2t, Di = CS.precond_blocks(KE, s.mass, s.gamma)
    M = np.block([[Bt, -At], [At, Bt]])
    r = np.random.default_rng(3).standard_normal(4 * s.n)
    exact = np.linalg.solve(M, r)
    assert np.linalg.norm(CS.precond_apply(KE, s.mass, s.gamma, r) - exact) <= 1e-10 * np.linalg.norm(exact)
    t = np.random.default_rng(4).standard_normal(2 * s.n)
    assert np.allclose(CS.s2t_solve(KE, s.mass, s.gamma, S2t @ t), t, atol=1e-8 * np.abs(t).max())
    n2 = 2 * s.n
    P = spla.LinearOperator((n2, n2), matvec=lambda v: CS.s2t_solve(KE, s.mass, s.gamma, v))
    SP = spla.LinearOperator((n2, n2), matvec=lambda v: S2 @ CS.s2t_solve(KE, s.mass, s.gamma, v))
    its = []
    y, info = spla.gmres(SP, t, rtol=1e-10, atol=0.0, restart=200, maxiter=1,
                         callback=lambda rk: its.append(rk), callback_type="pr_norm")
    w = P @ y
    assert info == 0 and np.linalg.norm(S2 @ w - t) <= 1e-9 * np.linalg.norm(t)
    assert len(its) <= 2 * s.k + 12
    # a splitting iteration w <- w + S2t^-1 (t - S2 w) does not converge here
    ws = np.zeros(n2)
    for _ in range(5):
        ws = ws + CS.s2t_solve(KE, s.mass, s.gamma, t - S2 @ ws)
    assert np.linalg.norm(S2 @ ws - t) > np.linalg.norm(t)
