"""Device storage of one solver, measured as the drop in free device memory
across `mrcg_solver_create`, against the library's own accounting.

Sec. 4, Table 2 counts the extra vectors MINRES-CG keeps besides A, M and b
as 11 + k (MINRES 7, CG 4, V_hat k).  This library keeps, besides the
operator and V_hat:
  * 9 FP64 outer vectors: x, b, the true residual, the raw and scaled inner
    solution at the precision boundary, v_j, v_{j+1}, w_j, w_{j+1};
  * 7 inner CG vectors in the inner precision: z, r, q and p twice (the fused
    SpMV writes p_i while gathering p_{i-1}), plus, with M_cg = I, a second r
    and q for the one-kernel iteration, or, with Jacobi, s and diag(M_mr)^{-1}.
That is 15 + k vectors besides A and b, every one of length n_pad = n rounded
up to 32 rows.  The test pins that nothing else of length n is allocated: an
unaccounted vector (32 MiB at this size) would exceed the bound, which leaves
2 MiB per small allocation and 8 MiB for the graphs."""
import numpy as np
import pytest

from gen import shifted_laplacian_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1805_12417_gb300 as m  # noqa: E402

MIB = 1 << 20
SLICE = 32           # SELL slice height
PARTIAL_SLOTS = (2 * (32 + 4) + 2) * 2048  # per-block reduction partials (FP64): step a's by parity, step b's


@pytest.fixture(scope="module")
def lap():
    # 2048^2 5-point Laplacian, n = 4,194,304: one FP64 vector is 32 MiB
    return shifted_laplacian_problem("storage", (2048, 2048), 4, seed=0)


def _accounted(p, fp32, mcg):
    """(large allocation sizes, number of small allocations) in bytes."""
    n, k = p.n, p.k
    nsl = (n + SLICE - 1) // SLICE
    n_pad = nsl * SLICE
    width = np.diff(p.rowptr)
    width = np.pad(width, (0, n_pad - n))
    total = int(width.reshape(nsl, SLICE).max(axis=1).sum()) * SLICE
    esz = 4 if fp32 else 8
    pad = 0  # allocations are exact
    large = [total * 4 + pad, total * 8 + pad, (total + 1) * 2 + pad, n_pad * k * 8 + pad]
    if fp32:
        large += [total * 4 + pad, n_pad * k * 4 + pad]
    large += [n_pad * 8 + pad] * 9
    large += [n_pad * esz + pad] * 7
    assert len(large) - (6 if fp32 else 4) - 1 + k == 15 + k  # vectors besides A, V_hat columns and b
    small = [(nsl + 1) * 8 + pad, PARTIAL_SLOTS * 8 + pad, 1, k * k * 8 + pad]
    return large, small


def _free():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("prec,mcg", [(m.FP64, m.MCG_IDENTITY), (m.MIXED_FP32, m.MCG_IDENTITY),
                                      (m.FP64, m.MCG_JACOBI)], ids=["fp64", "mixed", "fp64_jacobi"])
def test_solver_device_storage_is_accounted(lap, prec, mcg, monkeypatch):
    monkeypatch.setenv("MRCG_AUTOTUNE", "0")
    torch.zeros(1, device="cuda:0")
    kw = dict(precision=prec, inner_prec=mcg, validate=False)
    with m.Solver.from_problem(lap, **kw):  # loads the kernels' code first
        pass
    f0 = _free()
    with m.Solver.from_problem(lap, **kw):
        used = f0 - _free()
    large, small = _accounted(lap, prec == m.MIXED_FP32, mcg)
    lo = sum(large)
    hi = sum(-(-s // (2 * MIB)) * 2 * MIB for s in large) + 2 * MIB * len(small) + 8 * MIB
    print(f"device storage: {used / MIB:.1f} MiB, accounted {lo / MIB:.1f}..{hi / MIB:.1f} MiB")
    assert lo - MIB <= used <= hi, (used / MIB, lo / MIB, hi / MIB)
