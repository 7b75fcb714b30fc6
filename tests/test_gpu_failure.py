"""Failure detection on the GPU without a GPU fault.

The staged step-a kernels wait on mbarriers for their bulk copies; every wait
is bounded (about a second of clock), after which the block raises a shared
abort flag, waits (bounded) for the copies it did issue, and the solve reports
MRCG_ERR_CUDA.  MRCG_TEST_STALL=1 makes the producer stop issuing after the
first tile, so the consumers' waits on the next tile run out: a flag that
nothing sets.  The test checks the status and that the GPU context is still
usable afterwards (a fresh handle solves correctly).
"""
import time

import numpy as np
import pytest

import oracle as O
from gen import small_3d

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1805_12417_gb300 as m  # noqa: E402


@pytest.mark.parametrize("var", [5, 7, 14], ids=["staged", "pipelined", "twoslice"])
def test_stalled_copies_report_an_error_and_leave_the_context_usable(var, monkeypatch):
    p = small_3d()  # 6 tiles of 8 slices (3 of 16): block 0 has a second tile to wait for
    y = np.random.default_rng(2).standard_normal(p.n)
    monkeypatch.setenv("MRCG_VAR_A", str(var))
    monkeypatch.setenv("MRCG_STAGES", "2")
    monkeypatch.setenv("MRCG_TEST_STALL", "1")
    monkeypatch.setenv("MRCG_SHAPE_F64", f"{var},2,2,4")  # 2 blocks: each takes 3 tiles
    with m.Solver.from_problem(p) as g:
        assert m.launch_config(g.h)["step_a_variant"] == var
        t0 = time.perf_counter()
        with pytest.raises(m.MrcgError) as e:
            g.inner_solve(y, inner_tol=1e-8)
        dt = time.perf_counter() - t0
    assert e.value.status == m.ERR_CUDA
    assert dt < 30.0
    monkeypatch.delenv("MRCG_TEST_STALL")
    s = O.System.from_problem(p)
    zr, _, _ = s.cg(y, 1e-8, 100000, O.MCG_IDENTITY)
    with m.Solver.from_problem(p) as g:
        z, st, it = g.inner_solve(y, inner_tol=1e-8)
    assert st == m.OK
    assert np.linalg.norm(z - zr) <= 1e-8 * np.linalg.norm(zr)
