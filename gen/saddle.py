"""Saddle-point test systems [K B^T; B 0] with exactly nb negative eigenvalues.

Recipe (seeded, default_rng(seed), draws in this order):
  * K: graph Laplacian of the 27-point stencil on an m^3 grid (row index
    p + m*(q + m*r)); every undirected edge (a, b), a < b, in lexicographic
    (a, b) order gets a weight c_e ~ lognormal(0, 1); K_ab = K_ba = -c_e and
    K_aa = sum_b c_ab + 1 (strict diagonal dominance, so K is SPD with
    lambda_min(K) >= 1).
  * B: nb rows; row i takes nnzb distinct columns drawn uniformly from
    [0, m^3) and values uniform[-1, 1].
  * A = [[K, B^T], [B, 0]] (no stored zeros), n = m^3 + nb.  With K SPD and B
    of full row rank, A has exactly nb negative eigenvalues (Sylvester's law
    of inertia on the block LDL^T).
  * x* = uniform[-1, 1] (n values), b = A x*.
The negative eigenpairs (the paper's stage two, Sec. 2; MATLAB eigs there) are
computed by Rayleigh-Ritz on the block Krylov space of (K - shift I)^{-1} B^T
(dense eigh for small systems).  This module holds no MINRES-CG arithmetic.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .problems import Problem


def stencil27_laplacian(m: int, rng) -> sp.csr_matrix:
    n = m ** 3
    P, Q, R = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    P, Q, R = P.ravel(), Q.ravel(), R.ravel()
    a_all, b_all = [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dx == dy == dz == 0:
                    continue
                p2, q2, r2 = P + dx, Q + dy, R + dz
                ok = (p2 >= 0) & (p2 < m) & (q2 >= 0) & (q2 < m) & (r2 >= 0) & (r2 < m)
                a = (P + m * (Q + m * R))[ok]
                b = (p2 + m * (q2 + m * r2))[ok]
                keep = a < b
                a_all.append(a[keep]); b_all.append(b[keep])
    a = np.concatenate(a_all); b = np.concatenate(b_all)
    order = np.lexsort((b, a))
    a, b = a[order], b[order]
    w = rng.lognormal(0.0, 1.0, len(a))
    W = sp.coo_matrix((w, (a, b)), shape=(n, n)).tocsr()
    W = (W + W.T).tocsr()
    d = np.asarray(W.sum(axis=1)).ravel() + 1.0
    K = (sp.diags(d) - W).tocsr()
    K.sort_indices()
    return K


def saddle_matrix(m: int, nb: int, nnzb: int, seed: int):
    rng = np.random.default_rng(seed)
    K = stencil27_laplacian(m, rng)
    nK = K.shape[0]
    rows, cols, vals = [], [], []
    for i in range(nb):
        c = np.sort(rng.choice(nK, size=nnzb, replace=False))
        rows.append(np.full(nnzb, i)); cols.append(c); vals.append(rng.uniform(-1.0, 1.0, nnzb))
    B = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nb, nK))
    A = sp.bmat([[K, B.T], [B, None]], format="csr")
    A.sort_indices()
    A.eliminate_zeros()
    return A, K, B, rng


def _negative_eigenpairs_dense(A: sp.csr_matrix, nb: int):
    w, Q = np.linalg.eigh(A.toarray())
    return Q[:, :nb].copy(), w[:nb].copy()


def _negative_eigenpairs_krylov(K, B, nb, shift, blocks, cg_tol=1e-13, device=None):
    """Rayleigh-Ritz of A on span{[Y_j; 0], [0; I]}, Y_j an orthonormal block
    Krylov basis of (K - shift I)^{-1} applied to B^T (block CG solves).  Runs
    on the GPU when there is one (device None), else on the CPU (slowly)."""
    import torch

    if device is None:
        device = "cuda" if torch.cuda.is_available() else "cpu"
    dev = torch.device(device)
    nK = K.shape[0]
    Kt = torch.sparse_csr_tensor(torch.from_numpy(K.indptr.astype(np.int64)),
                                 torch.from_numpy(K.indices.astype(np.int64)),
                                 torch.from_numpy(K.data), size=K.shape, dtype=torch.float64).to(dev)

    def op(X):
        return torch.sparse.mm(Kt, X) - shift * X

    def solve(R):
        X = torch.zeros_like(R)
        Rr = R.clone()
        P = Rr.clone()
        rho = (Rr * Rr).sum(0)
        r0 = rho.sqrt()
        for _ in range(5000):
            AP = op(P)
            alpha = rho / (P * AP).sum(0)
            X += P * alpha
            Rr -= AP * alpha
            rho_new = (Rr * Rr).sum(0)
            if bool((rho_new.sqrt() <= cg_tol * r0).all()):
                break
            P = Rr + P * (rho_new / rho)
            rho = rho_new
        return X

    Bt = torch.from_numpy(B.toarray().T.copy()).to(dev)
    Qs = []
    Y = Bt
    for _ in range(blocks):
        Y = solve(Y)
        for _ in range(2):  # block Gram-Schmidt, twice
            for Qj in Qs:
                Y = Y - Qj @ (Qj.T @ Y)
        Y, _ = torch.linalg.qr(Y)
        Qs.append(Y)
    Q = torch.cat(Qs, dim=1)
    KQ = torch.sparse.mm(Kt, Q)
    H11 = (Q.T @ KQ).cpu().numpy()
    H12 = (Q.T @ Bt).cpu().numpy()
    s = Q.shape[1]
    H = np.zeros((s + nb, s + nb))
    H[:s, :s] = 0.5 * (H11 + H11.T)
    H[:s, s:] = H12
    H[s:, :s] = H12.T
    w, Z = np.linalg.eigh(H)
    Zt = torch.from_numpy(Z[:, :nb].copy()).to(dev)
    U = Q @ Zt[:s]
    V = torch.cat([U, Zt[s:]], dim=0).cpu().numpy()
    del Kt, Q, KQ, Qs
    torch.cuda.empty_cache()
    return V, w[:nb].copy()


def saddle_problem(m: int, nb: int = 20, nnzb: int = 64, seed: int = 2, shift: float = -0.75, blocks: int = 16,
                   name=None, dense_limit: int = 6000) -> Problem:
    A, K, B, rng = saddle_matrix(m, nb, nnzb, seed)
    n = A.shape[0]
    xstar = rng.uniform(-1.0, 1.0, n)
    b = A @ xstar
    if n <= dense_limit:
        V, lam = _negative_eigenpairs_dense(A, nb)
    else:
        V, lam = _negative_eigenpairs_krylov(K, B, nb, shift, blocks)
    res = np.linalg.norm(A @ V - V * lam, axis=0)
    meta = {"m": m, "nb": nb, "nnzb": nnzb, "seed": seed, "nK": K.shape[0], "eig_residual_max": float(res.max()),
            "lam_range": [float(lam.min()), float(lam.max())]}
    return Problem(name or f"saddle_{m}^3_B{nb}x{nnzb}", n, A.indptr.astype(np.int64), A.indices.astype(np.int32),
                   A.data.astype(np.float64), nb, V, lam, xstar, b, 0.0, meta)


def saddle_96_b20x64() -> Problem:
    """[K B^T; B 0], K 27-point log-normal on 96^3 (n = 884,756), B 20 x 64, seed 2."""
    return saddle_problem(96, 20, 64, seed=2, name="saddle_96^3_B20x64")


def small_saddle(m: int = 12, nb: int = 6, nnzb: int = 16, seed: int = 9) -> Problem:
    return saddle_problem(m, nb, nnzb, seed=seed)
