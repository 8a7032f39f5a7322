"""Mixed-precision sCholQR3 (CQR_PREC_MIXED): FP32 Gramian for the first,
shifted pass; FP64 norm estimate, Cholesky, solves and later passes.

The final factors are checked against the FP64 oracle with the same
tolerances as the FP64 path (test_gpu_factor.py): the first pass only
preconditions, the FP64 passes decide the result.  The first shift must be
the one sized for FP32 roundoff, 11 (n (2 u_in + d u_acc) + n (n+1) u) ||X||
with u_in = 2^-23, u_acc = 2^-24, d = 66.
"""
import numpy as np
import pytest

from paper_2507_07788_gb300 import synth
from parity import U, check_q, check_r

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cq():
    import paper_2507_07788_gb300 as cq
    from paper_2507_07788_gb300 import _build
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return cq



def mixed_coeff(n):
    u_in, u_acc = 2.0 ** -23, 2.0 ** -24
    return 11.0 * (n * (2 * u_in + 66 * u_acc) + n * (n + 1) * U)


@pytest.mark.parametrize("n", [64, 128])
@pytest.mark.parametrize("kappa", [1e6, 1e10, 1e14])
def test_mixed_parity(cq, orc, n, kappa):
    m = 40013
    A = synth.test_matrix(m, n, kappa, rep=4)
    dA = cq.to_colmajor(A)
    res = cq.factor(dA, opts=cq.default_opts(precision=cq.PREC_MIXED), check=False)
    ref = cq.factor(dA, check=False)
    torch.cuda.synchronize()
    Q, R = res.Q.cpu().numpy(), res.R.cpu().numpy()
    Qo, Ro, sto, info_o = orc.cholqr(A)
    assert res.status == cq.OK, res.info
    assert orc.loo_frob(Q) <= 1e-13
    assert orc.rrr(A, Q, R) <= 1e-13
    check_q(np.max(np.abs(Q - Qo)), kappa, m, f"mixed n={n} kappa={kappa:g}")
    check_r(np.max(np.abs(R - Ro)), kappa, Ro, m, f"mixed n={n} kappa={kappa:g}")
    # first shift sized for FP32 roundoff, from ||X|| (estimate within 1e-2)
    lam = orc.sym_norm2(orc.gram(A))
    assert res.info["sigma_first"] == pytest.approx(mixed_coeff(n) * lam, rel=2e-2)
    print(f"n={n} kappa={kappa:.0e} mixed iters={res.info['iters']} fp64 iters={ref.info['iters']} "
          f"loo={orc.loo_frob(Q):.2e}")


def test_mixed_orthonormal_input(cq):
    A = np.zeros((5000, 6))
    A[np.arange(6) * 7, np.arange(6)] = 1.0
    res = cq.factor(cq.to_colmajor(A), opts=cq.default_opts(precision=cq.PREC_MIXED))
    # the FP32 Gramian of an exactly orthonormal A is exact: no pass
    assert res.status == cq.OK and res.info["iters"] == 0
    assert np.array_equal(res.Q.cpu().numpy(), A)


def test_mixed_nan_breakdown(cq):
    A = synth.test_matrix(3000, 8, 10.0)
    A[9, 3] = np.nan
    res = cq.factor(cq.to_colmajor(A), opts=cq.default_opts(precision=cq.PREC_MIXED), check=False)
    assert res.status == cq.ERR_BREAKDOWN
