"""Seeded test problems with few negative eigenvalues.

The solver targets sparse, full-rank, symmetric indefinite A with k << n
negative eigenvalues (Sec. 1, Eq. 1).  The synthetic stand-ins are shifted
Dirichlet Laplacians A = L - sigma*I whose eigenpairs are known in closed form,
so the negative invariant subspace V_hat and its eigenvalues Lambda_hat
(Sec. 2, definition of M_mr) are exact up to rounding.

Recipe (one function per workload):
  * L: unscaled Dirichlet 5-point (2D) / 7-point (3D) stencil, row index
    p + m1*(q + m2*r) (x fastest); diagonal 2*d, off-diagonals -1.
  * eigenvalue of mode (i1, .., id): sum_d 2 - 2 cos(i_d pi / (m_d + 1)),
    eigenvector prod_d sqrt(2/(m_d+1)) sin(i_d pi (p_d+1) / (m_d+1)).
  * sigma midway between the k-th and (k+1)-th smallest eigenvalue; if they
    coincide (symmetric grids have degenerate clusters) k is raised to the end
    of its cluster so that A stays nonsingular.
  * x* = default_rng(seed).uniform(-1, 1, n); b = A x* (scipy CSR product).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class Problem:
    """One symmetric indefinite system with its negative eigenpairs.

    rowptr int64[n+1], colind int32[nnz], val float64[nnz]: full symmetric CSR
    with sorted column indices.  V float64[n, k] (C order, i.e. row-major; use
    V.T for the column-major n x k block the C-ABI takes), lam float64[k] < 0.
    """

    name: str
    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    val: np.ndarray
    k: int
    V: np.ndarray
    lam: np.ndarray
    xstar: np.ndarray
    b: np.ndarray
    sigma: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.colind, self.rowptr), shape=(self.n, self.n))

    def dense(self) -> np.ndarray:
        return self.scipy().toarray()

    def V_colmajor(self) -> np.ndarray:
        """V as one contiguous column-major n x k block (column j at offset j*n)."""
        return np.ascontiguousarray(self.V.T)


def laplacian_csr(dims, sigma: float = 0.0):
    """CSR of the Dirichlet Laplacian on a len(dims)-D grid, minus sigma*I."""
    dims = tuple(int(m) for m in dims)
    d = len(dims)
    n = int(np.prod(dims))
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for m in dims:
        coords.append(rem % m)
        rem //= m
    strides = [1]
    for m in dims[:-1]:
        strides.append(strides[-1] * m)
    rows = [idx]
    cols = [idx]
    vals = [np.full(n, 2.0 * d - sigma)]
    for ax, (m, st) in enumerate(zip(dims, strides)):
        lo = coords[ax] > 0
        rows.append(idx[lo]); cols.append(idx[lo] - st); vals.append(np.full(int(lo.sum()), -1.0))
        hi = coords[ax] < m - 1
        rows.append(idx[hi]); cols.append(idx[hi] + st); vals.append(np.full(int(hi.sum()), -1.0))
    r = np.concatenate(rows); c = np.concatenate(cols); v = np.concatenate(vals)
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, c.astype(np.int32), v.astype(np.float64)


def _mode_value(dims, modes):
    # sum of the per-axis values in sorted order, so that permuted modes of a
    # symmetric grid give bit-identical eigenvalues
    parts = sorted(2.0 - 2.0 * np.cos(i * np.pi / (m + 1)) for i, m in zip(modes, dims))
    s = 0.0
    for p in parts:
        s += p
    return s


def laplacian_smallest_eigs(dims, count: int):
    """The `count` smallest Laplacian eigenvalues with their mode tuples.

    Returned ascending with multiplicity; ties broken by the mode tuple.
    """
    dims = tuple(int(m) for m in dims)
    reach = 1
    while True:
        ranges = [range(1, min(m, reach) + 1) for m in dims]
        cand = [(_mode_value(dims, md), md) for md in itertools.product(*ranges)]
        cand.sort()
        if len(cand) > count:
            # every mode outside the box has some index > reach, so its value
            # exceeds the smallest value with that index: enlarge until the
            # count-th value is below that bound
            bound = min(_mode_value(dims, tuple(min(reach + 1, m) if a == ax else 1
                                                for a, m in enumerate(dims)))
                        for ax in range(len(dims)) if dims[ax] > reach) if any(m > reach for m in dims) else np.inf
            if cand[count][0] < bound:
                return cand[: count + 1]
        if all(m <= reach for m in dims):
            return cand
        reach += 2


def laplacian_eigvecs(dims, modes) -> np.ndarray:
    """Orthonormal eigenvectors (rows of the returned [len(modes), n] array)."""
    dims = tuple(int(m) for m in dims)
    out = np.empty((len(modes), int(np.prod(dims))))
    for t, md in enumerate(modes):
        vec = np.ones(1)
        for i, m in zip(modes[t], dims):
            axis = np.sqrt(2.0 / (m + 1)) * np.sin(i * np.pi * np.arange(1, m + 1) / (m + 1))
            vec = np.kron(axis, vec)  # x fastest
        out[t] = vec
    return out


def shift_for_negatives(dims, k_wanted: int, rel_tie: float = 1e-10):
    """sigma midway between eigenvalues k and k+1, with k raised past ties.

    Returns (sigma, k_eff, eigs[0:k_eff+1] as (value, mode)).
    """
    k = int(k_wanted)
    while True:
        ev = laplacian_smallest_eigs(dims, k + 1)
        lk, lk1 = ev[k - 1][0], ev[k][0]
        if abs(lk1 - lk) <= rel_tie * lk1:
            k += 1
            continue
        return 0.5 * (lk + lk1), k, ev[: k + 1]


def shifted_laplacian_problem(name, dims, k_wanted, seed, xstar=None, sigma_frac=0.5) -> Problem:
    """A = L - sigma I with sigma between eigenvalues k and k+1 of L: midway by
    default; sigma_frac < 0.5 puts it closer to lambda_k (negative eigenvalues
    of A closer to zero than the positive ones)."""
    sigma, k, ev = shift_for_negatives(dims, k_wanted)
    if sigma_frac != 0.5:
        sigma = ev[k - 1][0] + sigma_frac * (ev[k][0] - ev[k - 1][0])
    rowptr, colind, val = laplacian_csr(dims, sigma)
    n = int(np.prod(dims))
    modes = [m for _, m in ev[:k]]
    V = laplacian_eigvecs(dims, modes).T.copy()  # n x k, row-major
    lam = np.array([v for v, _ in ev[:k]]) - sigma
    if xstar is None:
        xstar = np.random.default_rng(seed).uniform(-1.0, 1.0, n)
    A = sp.csr_matrix((val, colind, rowptr), shape=(n, n))
    b = A @ xstar
    gap = min(abs(ev[k - 1][0] - sigma), abs(ev[k][0] - sigma))
    lam_max = sum(2.0 - 2.0 * np.cos(m * np.pi / (m + 1)) for m in dims) - sigma
    meta = {"dims": list(dims), "k_wanted": int(k_wanted), "k": k, "sigma": sigma,
            "min_abs_eig": gap, "max_abs_eig": lam_max, "cond": lam_max / gap, "seed": seed}
    return Problem(name, n, rowptr, colind, val, k, V, lam, xstar, b, sigma, meta)


def lap2d_64_k4() -> Problem:
    """2D 5-point Laplacian 64x64 (n=4096), 4 negative eigenvalues, seed 0."""
    return shifted_laplacian_problem("lap2d_64x64_k4", (64, 64), 4, seed=0)


def lap3d_128_k10() -> Problem:
    """3D 7-point Laplacian 128^3 (n=2,097,152), 10 negative eigenvalues, seed 1."""
    return shifted_laplacian_problem("lap3d_128^3_k10", (128, 128, 128), 10, seed=1)


def lap3d_128_k10_near() -> Problem:
    """The lap3d_128_k10 matrix with sigma moved to lambda_10 + 0.05 (lambda_11 - lambda_10):
    the 10 negative eigenvalues are the ones closest to zero (where the
    MINRES-CG* inner preconditioner of Sec. 2.1 pays off)."""
    return shifted_laplacian_problem("lap3d_128^3_k10_near", (128, 128, 128), 10, seed=1, sigma_frac=0.05)


def small_3d(m=(12, 11, 10), k=5, seed=7) -> Problem:
    """Small 3D analogue used by the parity tests (ragged in every dimension)."""
    return shifted_laplacian_problem(f"lap3d_{m[0]}x{m[1]}x{m[2]}_k{k}", m, k, seed=seed)


def random_indefinite_dense(n: int, k: int, seed: int, spread=(0.5, 4.0)):
    """Dense Q diag(d) Q^T with exactly k negative eigenvalues.

    Returns (A, V_neg[n,k], lam_neg[k], eigvals, Q).  Used only for tiny
    dense checks of the oracle.
    """
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    mags = rng.uniform(spread[0], spread[1], n)
    d = mags.copy()
    d[:k] = -mags[:k]
    A = (Q * d) @ Q.T
    A = 0.5 * (A + A.T)
    return A, Q[:, :k].copy(), d[:k].copy(), d, Q


def dense_to_csr(A: np.ndarray):
    """CSR (int64 rowptr, int32 colind, float64 values) of the nonzeros of A."""
    M = sp.csr_matrix(A)
    M.sort_indices()
    return M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64)


WORKLOADS = {
    "lap2d_64x64_k4": lap2d_64_k4,
    "lap3d_128^3_k10": lap3d_128_k10,
}


def random_sparse_symmetric(n: int, seed: int, density_rows=(0, 70), diag_shift: float = 0.0,
                            empty_rows: int = 2):
    """Random symmetric CSR with ragged row lengths (including empty rows).

    Off-diagonal pairs are drawn per row with a row-dependent count so that
    row lengths span density_rows; values uniform[-1, 1]; the diagonal is
    diag_shift plus uniform[-1, 1] except on `empty_rows` rows that keep no
    entry at all.  Used for the SpMV / M_mr product tests.
    """
    rng = np.random.default_rng(seed)
    lo, hi = density_rows
    rows, cols = [], []
    for i in range(n):
        cnt = int(rng.integers(lo, hi + 1)) // 2
        if cnt:
            js = rng.integers(0, n, cnt)
            rows.append(np.full(cnt, i)); cols.append(js)
    r = np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64)
    c = np.concatenate(cols) if cols else np.zeros(0, dtype=np.int64)
    v = rng.uniform(-1, 1, len(r))
    M = sp.coo_matrix((v, (r, c)), shape=(n, n)).tocsr()
    M = M + M.T
    M = M + sp.diags(diag_shift + rng.uniform(-1, 1, n))
    M = M.tolil()
    empties = rng.choice(n, size=min(empty_rows, n), replace=False)
    for e in empties:
        M[e, :] = 0
        M[:, e] = 0
    M = M.tocsr()
    M.eliminate_zeros()
    M.sort_indices()
    return M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64)


def batch64_lap2d(count: int = 64, sides=(100, 400), kmax: int = 16, seed: int = 3):
    """Batch of independent 2D 5-point Laplacian systems of uneven size.

    For each system i: square side m_i ~ U{sides}, then k_i ~ U{1..kmax}
    (raised to the end of its eigenvalue cluster), both drawn from
    default_rng(seed) in that order for all systems; then one right-hand side
    per system, uniform[-1, 1], from the same generator.  x* is unknown
    (xstar = None): the check is the true residual and the oracle solution.
    """
    rng = np.random.default_rng(seed)
    ms = rng.integers(sides[0], sides[1] + 1, size=count)
    ks = rng.integers(1, kmax + 1, size=count)
    out = []
    for i, (mi, ki) in enumerate(zip(ms, ks)):
        p = shifted_laplacian_problem(f"lap2d_{mi}x{mi}_k{ki}", (int(mi), int(mi)), int(ki), seed=None,
                                      xstar=np.zeros(int(mi) * int(mi)))
        out.append(p)
    for p in out:
        p.b = rng.uniform(-1.0, 1.0, p.n)
        p.xstar = None
    return out


@dataclass
class ShiftedFamily:
    """Shifted systems (L - sigma_j I) x = b sharing one sparsity pattern.

    L: CSR of the unshifted Laplacian; V: n x kmax eigenvectors of L (row
    index = unknown), lamL: their eigenvalues; sigma[j] and k[j] per shift;
    columns c = j * nrhs + r of B / xstar (n x ncols, C order) belong to
    shift j.  For column c the system is A = L - sigma_j I with
    V_hat = V[:, :k_j] and Lambda_hat = lamL[:k_j] - sigma_j.
    """

    name: str
    dims: tuple
    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    val: np.ndarray
    V: np.ndarray
    lamL: np.ndarray
    sigma: np.ndarray
    k: np.ndarray
    nrhs: int
    B: np.ndarray
    xstar: np.ndarray

    @property
    def ncols(self):
        return len(self.sigma) * self.nrhs

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def column_problem(self, c) -> Problem:
        """Column c as a stand-alone Problem (shifted CSR, its own V_hat / Lambda_hat)."""
        j = c // self.nrhs
        rp, ci, va = laplacian_csr(self.dims, self.sigma[j])
        kj = int(self.k[j])
        return Problem(f"{self.name}_col{c}", self.n, rp, ci, va, kj, self.V[:, :kj].copy(),
                       self.lamL[:kj] - self.sigma[j], self.xstar[:, c].copy(), self.B[:, c].copy(),
                       float(self.sigma[j]))


    def subfamily(self, shifts) -> "ShiftedFamily":
        """The family restricted to the listed shifts (their columns, in order;
        L shared, V and lamL cut to the largest k_j kept)."""
        shifts = [int(j) for j in shifts]
        cols = [j * self.nrhs + r for j in shifts for r in range(self.nrhs)]
        kmax = max(int(self.k[j]) for j in shifts)  # V and lamL trimmed to the widest shift kept
        return ShiftedFamily(f"{self.name}_shifts{'_'.join(map(str, shifts))}", self.dims, self.n, self.rowptr,
                             self.colind, self.val, np.ascontiguousarray(self.V[:, :kmax]), self.lamL[:kmax].copy(),
                             self.sigma[shifts].copy(),
                             self.k[shifts].copy(), self.nrhs, np.ascontiguousarray(self.B[:, cols]),
                             np.ascontiguousarray(self.xstar[:, cols]))


def shifted_family(dims, nshift, nrhs, kmax_draw, seed, name="shifted"):
    """k_j ~ U{1..kmax_draw} from default_rng(seed), each raised to the end of
    its eigenvalue cluster; sigma_j midway between eigenvalues k_j and k_j + 1
    of L; then x* for every (shift, rhs) column, uniform[-1, 1], from the same
    generator (column-major draw order: column c = j * nrhs + r)."""
    rng = np.random.default_rng(seed)
    kd = rng.integers(1, kmax_draw + 1, size=nshift)
    ks, sig = [], []
    for kw in kd:
        s, k, _ = shift_for_negatives(dims, int(kw))
        ks.append(k); sig.append(s)
    kmax = max(ks)
    ev = laplacian_smallest_eigs(dims, kmax + 1)
    lamL = np.array([v for v, _ in ev[:kmax]])
    V = laplacian_eigvecs(dims, [m for _, m in ev[:kmax]]).T.copy()
    rowptr, colind, val = laplacian_csr(dims)
    n = int(np.prod(dims))
    ncols = nshift * nrhs
    xs = np.empty((n, ncols))
    for c in range(ncols):
        xs[:, c] = rng.uniform(-1.0, 1.0, n)
    L = sp.csr_matrix((val, colind, rowptr), shape=(n, n))
    B = L @ xs
    sigc = np.repeat(np.array(sig), nrhs)
    B -= xs * sigc[None, :]
    return ShiftedFamily(name, tuple(dims), n, rowptr, colind, val, V, lamL, np.array(sig), np.array(ks), nrhs,
                         np.ascontiguousarray(B), xs)


def shifted_lap3d_160():
    """3D 7-point Laplacian 160^3, 16 shifts with k_j ~ U{1..30} (seed 4), 4 RHS each."""
    return shifted_family((160, 160, 160), 16, 4, 30, seed=4, name="lap3d_160^3_16shifts_x4")


def small_shifted(dims=(14, 13, 12), nshift=4, nrhs=2, kmax_draw=8, seed=5):
    return shifted_family(dims, nshift, nrhs, kmax_draw, seed, name=f"shifted_{dims[0]}x{dims[1]}x{dims[2]}")
