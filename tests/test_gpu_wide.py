"""Widths above 128 (up to CQR_MAX_N = 256): the FP64 row sweeps (the
Gramian split over several sweeps of its entries, the solve as a row-wise
substitution) and the control step on a global-memory working buffer.
Parity with the oracle by the bounds of tests/parity.py for the
factorisation at n = 129, 200 and 256, the Gramian at n = 256, an append of
160 columns to a basis of 64 (the oracle's Alg. 2 on its own basis of the
first block), and pnCholQR with 150-column panels (the oracle's Alg. 3); the
first width on the wide path, n = 129, beside the others."""
import numpy as np
import pytest

from paper_2507_07788_gb300 import synth
from parity import U, check_orth, check_q, check_r

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


@pytest.mark.parametrize("m,n,kappa", [(20011, 129, 1e6), (30007, 200, 1e10), (40013, 256, 1e12),
                                       (20011, 256, 1e4)])
def test_wide_factor_against_oracle(cq, orc, m, n, kappa):
    A = synth.test_matrix(m, n, kappa, rep=31)
    res = cq.factor(cq.to_colmajor(A), check=False)
    torch.cuda.synchronize()
    assert res.status == cq.OK, res.info
    Q, R = res.Q.cpu().numpy(), res.R.cpu().numpy()
    check_orth(Q, f"wide n={n}")
    assert orc.rrr(A, Q, R) <= 1e-13
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    Qo, Ro, sto, info_o = orc.cholqr(A)
    assert sto == cq.OK
    check_q(float(np.max(np.abs(Q - Qo))), kappa, m, f"wide n={n} kappa={kappa:g}")
    check_r(float(np.max(np.abs(R - Ro))), kappa, Ro, m, f"wide n={n} kappa={kappa:g}")
    # the first shift from the Gramian's norm (Alg. 1 line 6)
    lam = orc.sym_norm2(orc.gram(A))
    assert res.info["sigma_first"] == pytest.approx(orc.shift(m, n, lam), rel=1e-2)


def test_wide_gramian_against_oracle(cq, orc):
    m, n = 30011, 256
    A = synth.test_matrix(m, n, 1e8, rep=32)
    X = cq.gram(cq.to_colmajor(A)).cpu().numpy()
    Xo = orc.gram(A)
    absA = np.abs(A)
    bound = 2.0 * (m * U / (1 - m * U)) * (absA.T @ absA) + 1e-300
    assert np.all(np.abs(X - Xo) <= bound), float(np.max(np.abs(X - Xo) / bound))
    assert np.array_equal(X, X.T)


def test_wide_append_against_oracle(cq, orc):
    m, q, p = 20011, 64, 160
    rng = np.random.default_rng(33)
    A0 = synth.test_matrix(m, q, 1e4, rep=33)
    b = cq.Basis(m, q + p)
    st, _ = b.append(cq.to_colmajor(A0))
    assert st == cq.OK
    # the oracle's own basis of the same first block
    Qo0, Ro0, sto, _ = orc.cholqr(A0)
    assert sto == cq.OK
    blk = Qo0 @ rng.standard_normal((q, p)) * 0.1 + rng.standard_normal((m, p)) * 1e-3
    st, info = b.append(cq.to_colmajor(blk))
    assert st == cq.OK, info
    Q, R = b.Q().cpu().numpy(), b.R().cpu().numpy()
    b.close()
    check_orth(Q, "wide append")
    full = np.hstack([A0, blk])
    assert orc.rrr(full, Q, np.triu(R)) <= 1e-12
    # the oracle's Alg. 2 on its own basis
    Qn, Bn, Rn, sto, _ = orc.cholqr_update(Qo0, blk, min_iter=2)
    assert sto >= 0
    kap = float(np.linalg.cond(full))
    check_q(float(np.max(np.abs(Q[:, q:] - Qn))), kap, m, "wide append")
    Rnew = np.vstack([Bn, Rn])
    check_r(float(np.max(np.abs(R[: q + p, q:] - Rnew))), kap, Rnew, m, "wide append")


def test_wide_pn_panels(cq, orc):
    m, n, r, kappa = 20011, 300, 2, 1e6  # two panels of 150 columns
    A = synth.test_matrix(m, n, kappa, rep=34)
    res = cq.pn(cq.to_colmajor(A), r, check=False)
    torch.cuda.synchronize()
    assert res.status >= 0, res.status
    Q, R = res.Q.cpu().numpy(), res.R.cpu().numpy()
    check_orth(Q, "wide pn")
    assert orc.rrr(A, Q, R) <= 1e-12
    Qo, Ro, sto, _ = orc.pncholqr(A, r)
    assert sto >= 0
    check_q(float(np.max(np.abs(Q - Qo))), kappa, m, "wide pn")
    check_r(float(np.max(np.abs(R - Ro))), kappa, Ro, m, "wide pn")
