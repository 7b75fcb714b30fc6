"""GPU parity of the complex shifted systems of Sec. 3 (the disk-brake
application) on the synthetic stand-in of gen/brake.py: the solution of
(gamma B - A)(x + i y) = f + i g from the library's nested scheme (flexible
GMRES on the real-equivalent system, block-LU preconditioner, S2 by flexible
GMRES with S2t, MINRES-CG on KE - |gamma|^2 Mass) against the oracle's dense
complex solve (the definition), for two shifts of the same modulus on one
handle (the reuse Sec. 3 points out), with given and with computed
eigenpairs, in FP64 and mixed inner precision."""
import numpy as np
import pytest

from gen import brake_system, small_brake
from oracle import complex_shifted as CS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1805_12417_gb300 as m  # noqa: E402


def _relres(s, gamma, x, y):
    A, B = CS.companion(s.K.toarray(), s.D.toarray(), s.mass)
    C = gamma * B - A
    rhs = s.f + 1j * s.g
    return np.linalg.norm(rhs - C @ (x + 1j * y)) / np.linalg.norm(rhs)


@pytest.fixture(scope="module")
def small():
    return small_brake()


@pytest.mark.parametrize("given", [True, False], ids=["given_eigenpairs", "computed_eigenpairs"])
def test_two_shifts_of_one_modulus_match_the_dense_solve(small, given):
    s = small
    kw = {"V": s.V, "lam": s.lam} if given else {"eig_block": 16}
    with m.ComplexShifted(s, **kw) as cx:
        assert cx.negative_count == s.k
        for theta in (80.0, 60.0):
            g = abs(s.gamma) * np.exp(1j * np.deg2rad(theta))
            x, y, st, info = cx.solve(g, s.f, s.g, tol=1e-11)
            assert st == m.OK, info
            xr, yr = CS.complex_solve(s.K.toarray(), s.D.toarray(), s.mass, g, s.f, s.g)
            err = np.linalg.norm((x - xr) + 1j * (y - yr)) / np.linalg.norm(xr + 1j * yr)
            assert err <= 1e-8, (theta, err)
            assert _relres(s, g, x, y) <= 1e-10
            assert info["true_relres"] <= 1e-11 and info["inner_solves"] > 0


def test_mixed_inner_precision_reaches_the_tolerance(small):
    s = small
    with m.ComplexShifted(s, precision=m.MIXED_FP32, V=s.V, lam=s.lam) as cx:
        x, y, st, info = cx.solve(s.gamma, s.f, s.g, tol=1e-10)
    assert st == m.OK
    assert _relres(s, s.gamma, x, y) <= 1e-9


def test_device_arrays_and_a_wrong_modulus(small):
    s = small
    dev = torch.device("cuda:0")
    with m.ComplexShifted(s, V=s.V, lam=s.lam) as cx:
        x, y, st, info = cx.solve(s.gamma, torch.from_numpy(s.f).to(dev), torch.from_numpy(s.g).to(dev), tol=1e-10)
        assert st == m.OK
        assert _relres(s, s.gamma, x.cpu().numpy(), y.cpu().numpy()) <= 1e-9
        with pytest.raises(m.MrcgError) as e:
            cx.solve(1.1 * s.gamma, s.f, s.g)
        assert e.value.status == m.ERR_INVALID


def test_larger_stand_in_converges():
    """A 24^3 stand-in (n = 13,824; 55,296 real unknowns), k = 6, eigenpairs
    computed at create, mixed inner precision: the true relative residual of
    the complex system reaches 1e-8."""
    s = brake_system((24, 24, 24), 6, seed=13, name="brake_24^3_k6")
    with m.ComplexShifted(s, precision=m.MIXED_FP32, eig_block=24) as cx:
        assert cx.negative_count == s.k
        x, y, st, info = cx.solve(s.gamma, s.f, s.g, tol=1e-8, inner_tol=1e-6)
    assert st == m.OK and info["true_relres"] <= 1e-8
    print(f"brake 24^3: outer {info['outer_iters']}, S2 {info['s2_iters_total']}, inner solves "
          f"{info['inner_solves']}, CG {info['inner_cg_iters']}, {info['solve_ms']:.0f} ms")
