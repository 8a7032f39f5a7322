"""pnCholQR (Alg. 3, Sec. 2.3) on the GPU through cholqr_pn, against the
oracle's Alg. 3 with the same panel split (panel k has n/r columns, plus one
for k < n mod r).

Element-wise bounds are the QR perturbation bounds used for the
factorisation (about kappa u / sqrt(m) per entry of Q); orthogonality and the
residual are required to 1e-13 outright."""
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




@pytest.mark.parametrize("kappa", [1e4, 1e12])
@pytest.mark.parametrize("r", [1, 2, 3, 5, 40])
def test_pn_matches_oracle(cq, orc, kappa, r):
    m, n = 20037, 40
    A = synth.test_matrix(m, n, kappa, rep=31)
    res = cq.pn(cq.to_colmajor(A), r, check=False)
    torch.cuda.synchronize()
    Q, R = res.Q.cpu().numpy(), res.R.cpu().numpy()
    Qo, Ro, sto, info_o = orc.pncholqr(A, r)
    assert res.status == sto == cq.OK, (res.status, sto)
    assert orc.loo_frob(Q) <= 1e-13
    assert orc.rrr(A, Q, R) <= 1e-13
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    check_r(np.max(np.abs(R - Ro)), kappa, Ro, m, f"pn r={r} kappa={kappa:g}")
    check_q(np.max(np.abs(Q - Qo)), kappa, m, f"pn r={r} kappa={kappa:g}")
    # a panel sitting at a breakdown or stop threshold may take one pass
    # more or fewer on one side
    assert abs(res.info["iters"] - info_o.iters) <= r


def test_pn_single_panel_is_one_update(cq):
    # r = 1 is one Cholesky-QR update of an empty basis (Alg. 3 with one
    # panel): the same kernels as basis_append, so the same bits
    m, n = 9001, 24
    A = synth.test_matrix(m, n, 1e8, rep=32)
    dA = cq.to_colmajor(A)
    res = cq.pn(dA, 1)
    b = cq.Basis(m, n)
    b.append(dA)
    torch.cuda.synchronize()
    assert torch.equal(res.Q, b.Q()[:, :n]) and torch.equal(torch.triu(res.R), torch.triu(b.R()[:n, :n]))
    b.close()


def test_pn_and_factor_give_the_same_qr(cq, orc):
    # R is unique (positive diagonal), so pnCholQR and sCholQR3 agree up to
    # the perturbation bound
    m, n = 30011, 48
    A = synth.test_matrix(m, n, 1e6, rep=33)
    dA = cq.to_colmajor(A)
    rp = cq.pn(dA, 4)
    rf = cq.factor(dA)
    torch.cuda.synchronize()
    Rp, Rf = rp.R.cpu().numpy(), rf.R.cpu().numpy()
    check_r(np.max(np.abs(Rp - Rf)), 1e6, Rf, m, "pn vs factor")
    check_q(np.max(np.abs(rp.Q.cpu().numpy() - rf.Q.cpu().numpy())), 1e6, m, "pn vs factor")


def test_pn_zero_panel_not_converged_then_continues(cq, orc):
    # a zero panel (columns 16..23): its Gramian is 0, the shift floor 2u lets
    # every Cholesky succeed, Q stays 0 and the panel never converges; the
    # call reports NOT_CONVERGED (Alg. 2's loop ends at max_iter) and still
    # runs the later panels, as the oracle does
    m, n = 5000, 32
    A = synth.test_matrix(m, n, 1e3, rep=34)
    A[:, 16:24] = 0.0
    res = cq.pn(cq.to_colmajor(A), 4, check=False)
    Qo, Ro, sto, info_o = orc.pncholqr(A, 4)
    assert res.status == sto == cq.NOT_CONVERGED
    Q = res.Q.cpu().numpy()
    # the last panel was still appended, orthogonal to the first two
    assert np.max(np.abs(Q[:, :16].T @ Q[:, 24:])) <= 1e-13


def test_pn_nan_panel_breaks_down_and_stops(cq, orc):
    m, n = 5000, 32
    A = synth.test_matrix(m, n, 1e3, rep=35)
    A[17, 20] = np.nan
    res = cq.pn(cq.to_colmajor(A), 4, check=False)
    Qo, Ro, sto, info_o = orc.pncholqr(A, 4)
    assert res.status == sto == cq.ERR_BREAKDOWN


@pytest.mark.parametrize("r", [1, 3])
def test_pn_tall_matches_oracle(cq, orc, r):
    # m above the batched-append rows: the first panel (an append to an empty
    # basis) runs the tensor-core pass pipeline, later panels the update path
    m, n = 300007, 48
    A = synth.test_matrix(m, n, 1e10, rep=36)
    dA = cq.to_colmajor(A)
    res = cq.pn(dA, r, check=False)
    torch.cuda.synchronize()
    Q, R = res.Q.cpu().numpy(), res.R.cpu().numpy()
    Qo, Ro, sto, info_o = orc.pncholqr(A, r)
    assert res.status == sto == cq.OK, (res.status, sto)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 1e-13
    assert orc.rrr(A, Q, R) <= 1e-13
    check_r(np.max(np.abs(R - Ro)), 1e10, Ro, m, f"pn tall n={n}")
    check_q(np.max(np.abs(Q - Qo)), 1e10, m, f"pn tall n={n}")
