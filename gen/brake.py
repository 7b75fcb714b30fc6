"""Synthetic stand-in for the disk-brake systems of Sec. 3 (the finite
element matrices of the paper are not available).

Recipe (seeded, default_rng(seed), draws in this order), on an m1 x m2 x m3
grid (n = m1 m2 m3 mechanical unknowns):
  * KE: the 7-point Dirichlet Laplacian (symmetric positive definite
    stiffness);
  * Mass: lumped (diagonal) mass, the constant mass0 (a uniform grid with a
    uniform density);
  * KR: a general (nonsymmetric) perturbation on the stencil's off-diagonal
    pattern, eps_k * uniform[-1, 1] drawn independently for (i, j) and (j, i);
    K = KE + KR plays K_Omega;
  * D = alpha Mass + beta KE + DG with DG skew-symmetric on the same pattern
    (delta * uniform[-1, 1] per edge, i < j, and its negative at (j, i));
    D plays D_Omega;
  * the shift gamma = |gamma| (cos theta + i sin theta), with |gamma|^2 Mass
    midway between the k-th and (k+1)-th eigenvalues of KE (analytic), so the
    inner-level matrix KE - |gamma|^2 Mass has exactly k negative eigenvalues
    (rounded up to the end of a degenerate cluster, as for the shifted
    Laplacians);
  * f, g: uniform[-1, 1], 2n entries each.
This module holds no solver arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .problems import laplacian_csr, laplacian_eigvecs, shift_for_negatives


@dataclass
class BrakeSystem:
    name: str
    dims: tuple
    n: int
    KE: sp.csr_matrix
    K: sp.csr_matrix
    D: sp.csr_matrix
    mass: np.ndarray
    gamma: complex
    k: int
    V: np.ndarray      # n x k eigenvectors of KE - |gamma|^2 Mass with negative eigenvalues (analytic)
    lam: np.ndarray    # their eigenvalues
    f: np.ndarray
    g: np.ndarray

    @staticmethod
    def csr_arrays(M):
        M = M.tocsr()
        M.sort_indices()
        return M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64)


def _edges(KE):
    C = sp.triu(KE, k=1).tocoo()
    return C.row, C.col


def brake_system(dims, k_wanted, seed, mass0=1e-3, eps_k=0.02, alpha=0.05, beta=0.01, delta=0.05,
                 theta_deg=80.0, name="brake") -> BrakeSystem:
    rng = np.random.default_rng(seed)
    rp, ci, va = laplacian_csr(dims)
    n = int(np.prod(dims))
    KE = sp.csr_matrix((va, ci, rp), shape=(n, n))
    mass = np.full(n, mass0)
    a, b = _edges(KE)
    kr_ab = eps_k * rng.uniform(-1.0, 1.0, len(a))
    kr_ba = eps_k * rng.uniform(-1.0, 1.0, len(a))
    KR = sp.coo_matrix((np.concatenate([kr_ab, kr_ba]), (np.concatenate([a, b]), np.concatenate([b, a]))),
                       shape=(n, n)).tocsr()
    dg = delta * rng.uniform(-1.0, 1.0, len(a))
    DG = sp.coo_matrix((np.concatenate([dg, -dg]), (np.concatenate([a, b]), np.concatenate([b, a]))),
                       shape=(n, n)).tocsr()
    K = (KE + KR).tocsr()
    D = (alpha * sp.diags(mass) + beta * KE + DG).tocsr()
    # |gamma|^2 mass0 midway between eigenvalues k and k+1 of KE (cluster-rounded k)
    sigma, k, ev = shift_for_negatives(dims, k_wanted)
    mod2 = sigma / mass0
    th = np.deg2rad(theta_deg)
    gamma = complex(np.sqrt(mod2) * np.cos(th), np.sqrt(mod2) * np.sin(th))
    lam = np.array([v for v, _ in ev[:k]]) - sigma
    V = laplacian_eigvecs(dims, [md for _, md in ev[:k]]).T.copy()
    f = rng.uniform(-1.0, 1.0, 2 * n)
    g = rng.uniform(-1.0, 1.0, 2 * n)
    for M in (KE, K, D):
        M.sort_indices()
    return BrakeSystem(name, tuple(dims), n, KE, K, D, mass, gamma, k, V, lam, f, g)


def small_brake():
    return brake_system((9, 8, 7), 4, seed=11, name="brake_9x8x7_k4")


def brake_64():
    """The benchmark-size stand-in: a 64^3 grid (n = 262,144 mechanical
    unknowns, 1,048,576 in the real-equivalent system), k = 10."""
    return brake_system((64, 64, 64), 10, seed=12, name="brake_64^3_k10")
