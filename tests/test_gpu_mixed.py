"""Mixed-precision sCholQR3 (CQR_PREC_MIXED): a reduced-precision Gramian for
the first, shifted pass; FP64 norm estimate, Cholesky, solves and later
passes.

With the digit kernels (the default) the first Gramian keeps 5 balanced
base-256 digits of each element and the digit orders <= 4; a row adds at most
e Ubar_i Ubar_j to X_ij (e = 2.0324e-12, Ubar_j = 2^(E_j - 1022) for column
j's largest biased exponent), and the first shift is
  11 (m e sum_j Ubar_j^2 + n (n + 1 + G + 9) u ||X||).
The Gramian is checked against that bound entry by entry: against the
oracle's Gramian on the test matrices, and against the exact (integer)
Gramian of an adversarial matrix whose dropped digits are all at their
largest, where the error adds up coherently over the rows and comes within
a small factor of the bound.  With CQR_EMU_OFF the first Gramian is the FP32
sweep and the shift is 11 (n (2 u_in + d u_acc) + n (n+1) u) ||X|| with
u_in = 2^-23, u_acc = 2^-24, d = 66.

The final factors are checked against the FP64 oracle with the bounds of the
FP64 path (tests/parity.py): the first pass only preconditions, the FP64
passes decide the result.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2507_07788_gb300 import synth
from parity import MIXED_ROW_ERR, U, check_q, check_r, mixed_shift_terms, record, ubar

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


def fp32_coeff(n):
    u_in, u_acc = 2.0 ** -23, 2.0 ** -24
    return 11.0 * (n * (2 * u_in + 66 * u_acc) + n * (n + 1) * U)


def partials_max():
    return 2 * torch.cuda.get_device_properties(0).multi_processor_count


def gram_bound(A, partials):
    """Entry bound of |X_mixed - X|: m rows of e Ubar_i Ubar_j, plus the
    rounding of the partials and their sum ((G + 10) u sqrt(X_ii X_jj))."""
    m = A.shape[0]
    ub = ubar(A)
    d = np.sqrt(np.sum(A * A, axis=0))
    return m * MIXED_ROW_ERR * np.outer(ub, ub) + (partials + 10) * U * np.outer(d, d)


@pytest.mark.parametrize("n", [8, 40, 72, 128])
@pytest.mark.parametrize("kappa", [1e2, 1e10])
def test_mixed_gramian_within_its_bound(cq, orc, n, kappa):
    m = 50021
    A = synth.test_matrix(m, n, kappa, rep=5)
    dA = cq.to_colmajor(A)
    Xm = cq.gram(dA, opts=cq.default_opts(precision=cq.PREC_MIXED)).cpu().numpy()
    Xo = orc.gram(A)
    absA = np.abs(A)
    bound = gram_bound(A, partials_max()) + 2.0 * m * U * (absA.T @ absA)  # + the oracle's own error
    err = np.abs(Xm - Xo)
    record("mixed Gramian (max |dX| / bound)", float(np.max(err / bound)), 1.0, f"n={n} kappa={kappa:g}")
    assert np.all(err <= bound), float(np.max(err / bound))
    assert np.array_equal(Xm, Xm.T)


def adversarial(m, n, seed):
    """x = V 2^-56 with V = h 2^16 + 0x7F78, h random in [2^39, 2^40): every
    element in [1/2, 1) (Ubar = 1), its two dropped balanced digits 127 and
    120 (the largest a double's 53-bit mantissa allows), all positive."""
    rng = np.random.default_rng(seed)
    h = rng.integers(1 << 39, 1 << 40, size=(m, n), dtype=np.int64)
    V = (h << 16) | 0x7F78
    return V, np.ldexp(V.astype(np.float64), -56)


def exact_gram(V):
    """sum_r V_ri V_rj 2^-112 exactly (Python integers), rounded once to FP64."""
    m, n = V.shape
    hi, lo = V >> 28, V & ((1 << 28) - 1)
    acc = [[0] * n for _ in range(n)]
    for r0 in range(0, m, 64):  # 64 products of < 2^56 stay below 2^62
        h, l = hi[r0:r0 + 64], lo[r0:r0 + 64]
        hh, hl, ll = h.T @ h, h.T @ l, l.T @ l
        for i in range(n):
            for j in range(n):
                acc[i][j] += (int(hh[i, j]) << 56) + ((int(hl[i, j]) + int(hl[j, i])) << 28) + int(ll[i, j])
    return np.array([[float(Fraction(acc[i][j], 1 << 112)) for j in range(n)] for i in range(n)])


@pytest.mark.parametrize("n", [8, 64])
def test_mixed_gramian_adversarial_digits(cq, n):
    m = 20480
    V, A = adversarial(m, n, seed=n)
    assert np.array_equal(np.ldexp(A, 56).astype(np.int64), V)  # the elements are exact
    X = exact_gram(V)
    Xm = cq.gram(cq.to_colmajor(A), opts=cq.default_opts(precision=cq.PREC_MIXED)).cpu().numpy()
    bound = gram_bound(A, partials_max())
    err = np.abs(Xm - X)
    ratio = float(np.max(err / bound))
    record("mixed Gramian, adversarial digits (max |dX| / bound)", ratio, 1.0, f"n={n}")
    assert np.all(err <= bound), ratio
    # the truncation is in effect and adds up coherently: the error is well
    # above FP64 rounding and within a factor ~10 of the bound
    assert ratio > 0.05, ratio
    assert np.all(Xm <= X)  # dropped digits of positive elements are positive: X is underestimated
    # the FP64 (7-digit) Gramian of the same matrix is exact up to the
    # rounding of the partials and their fixed-order sum: hundreds of times
    # closer than the reduced one
    Xf = cq.gram(cq.to_colmajor(A)).cpu().numpy()
    ef = np.abs(Xf - X)
    assert np.all(ef <= (partials_max() + 12) * U * np.abs(X))
    assert np.max(ef) * 100 <= np.max(err), (float(np.max(ef)), float(np.max(err)))


@pytest.mark.parametrize("emulation", ["auto", "off"])
@pytest.mark.parametrize("n", [64, 128])
@pytest.mark.parametrize("kappa", [1e6, 1e10, 1e14])
def test_mixed_parity(cq, orc, n, kappa, emulation):
    m = 40013
    A = synth.test_matrix(m, n, kappa, rep=4)
    dA = cq.to_colmajor(A)
    emu = cq.EMU_AUTO if emulation == "auto" else cq.EMU_OFF
    res = cq.factor(dA, opts=cq.default_opts(precision=cq.PREC_MIXED, emulation=emu), check=False)
    ref = cq.factor(dA, check=False)
    torch.cuda.synchronize()
    Q, R = res.Q.cpu().numpy(), res.R.cpu().numpy()
    Qo, Ro, sto, info_o = orc.cholqr(A)
    assert res.status == cq.OK, res.info
    assert orc.loo_frob(Q) <= 1e-13
    assert orc.rrr(A, Q, R) <= 1e-13
    check_q(np.max(np.abs(Q - Qo)), kappa, m, f"mixed {emulation} n={n} kappa={kappa:g}")
    check_r(np.max(np.abs(R - Ro)), kappa, Ro, m, f"mixed {emulation} n={n} kappa={kappa:g}")
    # the first shift (from ||X||, estimated within 1e-2)
    lam = orc.sym_norm2(orc.gram(A))
    s1 = res.info["sigma_first"]
    if emulation == "off":
        assert s1 == pytest.approx(fp32_coeff(n) * lam, rel=2e-2)
    else:
        lo, hi = mixed_shift_terms(A, lam, partials_max())
        assert 0.98 * lo <= s1 <= 1.02 * hi, (s1, lo, hi)
        # at this m the two first shifts are of one size (the FP64 one grows
        # with m, this one does not): at most one pass more than FP64
        assert res.info["iters"] <= ref.info["iters"] + 1, (res.info, ref.info)
    print(f"n={n} kappa={kappa:.0e} {emulation}: mixed iters={res.info['iters']} "
          f"fp64 iters={ref.info['iters']} sigma1/||X||={s1 / lam:.2e} loo={orc.loo_frob(Q):.2e}")


@pytest.mark.parametrize("emulation", ["auto", "off"])
def test_mixed_orthonormal_input(cq, emulation):
    A = np.zeros((5000, 6))
    A[np.arange(6) * 7, np.arange(6)] = 1.0
    emu = cq.EMU_AUTO if emulation == "auto" else cq.EMU_OFF
    res = cq.factor(cq.to_colmajor(A), opts=cq.default_opts(precision=cq.PREC_MIXED, emulation=emu))
    # the reduced Gramian of an exactly orthonormal A is exact: no pass
    assert res.status == cq.OK and res.info["iters"] == 0
    assert np.array_equal(res.Q.cpu().numpy(), A)


@pytest.mark.parametrize("emulation", ["auto", "off"])
def test_mixed_nan_breakdown(cq, emulation):
    A = synth.test_matrix(3000, 8, 10.0)
    A[9, 3] = np.nan
    emu = cq.EMU_AUTO if emulation == "auto" else cq.EMU_OFF
    res = cq.factor(cq.to_colmajor(A), opts=cq.default_opts(precision=cq.PREC_MIXED, emulation=emu),
                    check=False)
    assert res.status == cq.ERR_BREAKDOWN
