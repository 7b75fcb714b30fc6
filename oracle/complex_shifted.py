"""Dense reference for the complex shifted systems of Sec. 3 (disk-brake
application): C (x + i y) = f + i g with C = gamma B - A, where A, B are the
companion linearisation of the quadratic pencil
    lambda^2 Mass + lambda D + K,   A = [[0, I], [-K, -D]], B = [[I, 0], [0, Mass]],
rewritten as the double-size real system (Sec. 3, the real-equivalent form)
    [[Bh, -Ah], [Ah, Bh]] [x; -y] = [g; f],
    Ah = [[gr I, -I], [K, gr Mass + D]],  Bh = [[gi I, 0], [0, gi Mass]],
and preconditioned by M = [[Bt, -At], [At, Bt]] with At = [[gr I, -I], [KE, gr Mass]]
and Bt = Bh, whose block LU uses the Schur complement S = Bt + At Bt^-1 At =
S1 S2 (S1 = diag(Mass^-1, I)), and S2 is approximated by its block lower
triangular part S2t whose diagonal blocks are -(1/gi) (KE - |gamma|^2 Mass):
the inner-level system MINRES-CG solves.

TEST INFRASTRUCTURE ONLY (small dense matrices).  Plain numpy, written from
the section's formulas in their order; nothing here is shared with the CUDA
library.  Mass is the lumped (diagonal) mass matrix, given as a vector.
"""
from __future__ import annotations

import numpy as np


def companion(K, D, mass):
    """A and B of the companion linearisation (2n x 2n, dense)."""
    n = K.shape[0]
    I = np.eye(n)
    Z = np.zeros((n, n))
    A = np.block([[Z, I], [-K, -D]])
    B = np.block([[I, Z], [Z, np.diag(mass)]])
    return A, B


def complex_solve(K, D, mass, gamma, f, g):
    """The definition: (gamma B - A) (x + i y) = f + i g by a dense complex solve.
    Returns (x, y), each of length 2n."""
    A, B = companion(K, D, mass)
    C = gamma * B - A
    z = np.linalg.solve(C, f + 1j * g)
    return z.real.copy(), z.imag.copy()


def real_blocks(K, D, mass, gamma):
    """Ah, Bh with C = Ah + i Bh (Sec. 3)."""
    n = K.shape[0]
    gr, gi = gamma.real, gamma.imag
    I = np.eye(n)
    Mm = np.diag(mass)
    Ah = np.block([[gr * I, -I], [K, gr * Mm + D]])
    Bh = np.block([[gi * I, np.zeros((n, n))], [np.zeros((n, n)), gi * Mm]])
    return Ah, Bh


def real_equivalent(K, D, mass, gamma):
    """The 4n x 4n real system [[Bh, -Ah], [Ah, Bh]] acting on [x; -y]."""
    Ah, Bh = real_blocks(K, D, mass, gamma)
    return np.block([[Bh, -Ah], [Ah, Bh]])


def precond_blocks(KE, mass, gamma):
    """At, Bt of the preconditioner and the pieces of its Schur complement:
    S = Bt + At Bt^-1 At, S1 = diag(Mass^-1, I), S2, and the block lower
    triangular S2t; Di = c Mass - KE / gi with c = gi + gr^2 / gi (the
    diagonal block of S2), so that S2t's diagonal solves are Di^-1."""
    n = KE.shape[0]
    gr, gi = gamma.real, gamma.imag
    I = np.eye(n)
    Mm = np.diag(mass)
    At = np.block([[gr * I, -I], [KE, gr * Mm]])
    Bt = np.block([[gi * I, np.zeros((n, n))], [np.zeros((n, n)), gi * Mm]])
    S = Bt + At @ np.linalg.solve(Bt, At)
    S1 = np.block([[np.diag(1.0 / mass), np.zeros((n, n))], [np.zeros((n, n)), I]])
    c = gi + gr * gr / gi
    Di = c * Mm - KE / gi
    S2 = np.block([[Di, -2.0 * gr / gi * Mm], [2.0 * gr / gi * KE, Di]])
    S2t = np.block([[Di, np.zeros((n, n))], [2.0 * gr / gi * KE, Di]])
    return At, Bt, S, S1, S2, S2t, Di


def inner_level_matrix(KE, mass, gamma):
    """KE - |gamma|^2 Mass, the symmetric inner-level matrix (Sec. 3): Di = -(1/gi) times it."""
    return KE - abs(gamma) ** 2 * np.diag(mass)


def s2t_solve(KE, mass, gamma, a):
    """S2t^-1 a (block forward substitution): t1 = Di^-1 a1,
    t2 = Di^-1 (a2 - 2 (gr/gi) KE t1), with Di^-1 v = -gi (KE - |gamma|^2 Mass)^-1 v."""
    n = KE.shape[0]
    gr, gi = gamma.real, gamma.imag
    Ain = inner_level_matrix(KE, mass, gamma)
    t1 = -gi * np.linalg.solve(Ain, a[:n])
    t2 = -gi * np.linalg.solve(Ain, a[n:] - 2.0 * gr / gi * (KE @ t1))
    return np.concatenate([t1, t2])


def precond_apply(KE, mass, gamma, r):
    """M^-1 r by the block LU of M (Sec. 3), every block solve exact:
      w1 = Bt^-1 r1;  t = r2 - At w1;  w2 = S^-1 t = S2^-1 (S1^-1 t);
      u2 = w2;  u1 = w1 + Bt^-1 At u2.   (r has 4n entries)"""
    n = KE.shape[0]
    At, Bt, S, S1, S2, S2t, Di = precond_blocks(KE, mass, gamma)
    r1, r2 = r[: 2 * n], r[2 * n:]
    w1 = np.linalg.solve(Bt, r1)
    t = r2 - At @ w1
    t = np.concatenate([mass * t[:n], t[n:]])  # S1^-1 t
    w2 = np.linalg.solve(S2, t)
    u2 = w2
    u1 = w1 + np.linalg.solve(Bt, At @ u2)
    return np.concatenate([u1, u2])
