"""MRCG_MIXED_BF16M: the mixed solver with V_hat's values rounded to BF16.

The rounding happens once, at create (round to nearest even from the FP32
value), and every inner kernel then computes with the rounded V_hat, so M_mr
(Eq. 5) is built on it.  Pins: (1) against the mixed solver given the same
rounded V_hat in FP32 the results are bitwise equal (the one-gather step a on
16-slice tiles streams BF16 bits and widens them exactly); (2) against the
FP64 oracle run on the rounded V_hat, x agrees within the solve tolerance;
(3) at 128^3 the solve reaches the benchmark tolerance with about the same
inner iterations as the FP32 V_hat.  The rounding rule itself is pinned on
the CPU against torch's bfloat16 conversion."""
import numpy as np
import pytest

import oracle as O
from gen import lap3d_128_k10, shifted_laplacian_problem

torch = pytest.importorskip("torch")

SHAPE = "14,2,304,152"  # one-gather step a on 16-slice tiles, 2 stages


def bf16_round(V):
    """V (FP64) -> FP64 values of BF16 numbers: FP32 first, then the upper 16
    bits after rounding the lower 16 to nearest, ties to even."""
    u = np.ascontiguousarray(V, dtype=np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_rounding_rule_is_round_to_nearest_even():
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(20000), rng.uniform(-1e-3, 1e-3, 20000),
                        # exact ties between two BF16 neighbours, both parities
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 0.0])])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(bf16_round(x), ref)
    assert bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0  # tie to the even neighbour
    assert bf16_round(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6


gpu = pytest.mark.gpu
needs_cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def _m():
    import paper_1805_12417_gb300 as m
    return m


def _problem():
    # 41^3 = 68,921 rows: 135 tiles of 512 rows, the last one ragged
    return shifted_laplacian_problem("bf16_41", (41, 41, 41), 10, seed=7)


@gpu
@needs_cuda
def test_bf16_equals_fp32_on_the_rounded_vhat(monkeypatch):
    m = _m()
    monkeypatch.setenv("MRCG_SHAPE_F32", SHAPE)
    p = _problem()
    Vr = bf16_round(p.V)
    out = []
    for prec, V in ((m.MIXED_BF16M, p.V), (m.MIXED_FP32, Vr)):
        with m.Solver(p.n, p.rowptr, p.colind, p.val, V, p.lam, precision=prec, validate=False) as g:
            assert m.launch_config(g.h)["step_a_variant"] == 14
            x, info = g.solve(p.b.copy(), outer_tol=1e-11, inner_tol=1e-3)
        assert info.status == m.OK
        out.append((x, info.outer_iters, info.inner_iters_total))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1:] == out[1][1:]


@gpu
@needs_cuda
@pytest.mark.parametrize("shape", [SHAPE, None], ids=["variant14", "autotuned"])
def test_bf16_matches_the_oracle_on_the_rounded_vhat(shape, monkeypatch):
    m = _m()
    if shape:
        monkeypatch.setenv("MRCG_SHAPE_F32", shape)
    p = _problem()
    Vr = bf16_round(p.V)
    with m.Solver(p.n, p.rowptr, p.colind, p.val, p.V, p.lam, precision=m.MIXED_BF16M) as g:
        x, info = g.solve(p.b.copy(), outer_tol=1e-12, inner_tol=1e-3)
    assert info.status == m.OK
    s = O.System(p.rowptr, p.colind, p.val, np.ascontiguousarray(Vr), p.lam)
    ref = O.minres_cg(s, p.b, outer_tol=1e-12, inner_tol=1e-3)
    assert ref.status == O.OK
    assert s.true_relres(p.b, x) <= 1e-12
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
    assert np.linalg.norm(x - p.xstar) <= 1e-8 * np.linalg.norm(p.xstar)


@gpu
@needs_cuda
def test_bf16_full_size_reaches_the_benchmark_tolerance():
    m = _m()
    p = lap3d_128_k10()
    res = {}
    for prec in (m.MIXED_FP32, m.MIXED_BF16M):
        with m.Solver.from_problem(p, precision=prec, validate=False) as g:
            x = torch.zeros(p.n, dtype=torch.float64, device="cuda:0")
            _, info = g.solve(torch.from_numpy(p.b).to("cuda:0"), x, outer_tol=1e-10, inner_tol=1e-3)
            res[prec] = (info, x.cpu().numpy(), m.launch_config(g.h)["step_a_variant"])
    info, x, var = res[m.MIXED_BF16M]
    assert info.status == m.OK and info.true_relres <= 1e-10
    assert np.linalg.norm(x - p.xstar) <= 1e-8 * np.linalg.norm(p.xstar)
    assert info.inner_iters_total <= 1.1 * res[m.MIXED_FP32][0].inner_iters_total
    print(f"bf16 V_hat 128^3: variant {var}, outer {info.outer_iters}, inner {info.inner_iters_total} "
          f"(FP32 V_hat: {res[m.MIXED_FP32][0].inner_iters_total})")


@gpu
@needs_cuda
def test_batch_and_shifted_handles_reject_bf16():
    m = _m()
    p = shifted_laplacian_problem("b", (21, 19), 3, seed=1)
    with pytest.raises(m.MrcgError) as e:
        m.Batch([p, p], precision=m.MIXED_BF16M)
    assert e.value.status == m.ERR_INVALID
