"""Widths above 128 (up to CQR_MAX_N = 512).  The Gramian is formed by
64 x 64 block pairs on the tensor cores and the
solve Q = Y T (T = D R~^{-1}) on the tensor cores with the contraction in
blocks of 64 (exact digit products; with CQR_EMU_OFF the FP64 row sweeps:
the Gramian split over several sweeps of its entries, the row-wise
substitution), and the control step works on a global-memory copy of the
n x n Gramian whose Cholesky is shared by the CTAs of a cooperative launch
(panels of 64 columns, grid barriers in between).  Parity with
the oracle by the bounds of tests/parity.py for the factorisation at n = 129,
200, 256, 300 and 512 (both Gramians), the Gramian at n = 256 and 512
(against the oracle's, and exactly on integer data whose Gramian FP64 holds
without rounding, which any misplaced or dropped block fails), an append of
160 columns to a basis of 64 (the oracle's Alg. 2 on its own basis of the
first block), an append of 300 columns to an empty basis, and pnCholQR with
150-column panels (the oracle's Alg. 3); the in-place factorisation equals
the out-of-place one bit for bit; a failing pivot, the recomputed shift and
the retry match the oracle's counters; the mixed variant, two row-sharded
ranks, and two concurrent factorisations on two streams (whose cooperative
steps take turns on the device's cooperative stream)."""
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


@pytest.mark.parametrize("emulation", ["auto", "off"])
@pytest.mark.parametrize("m,n,kappa", [(20011, 129, 1e6), (30007, 200, 1e10), (40013, 256, 1e12),
                                       (20011, 256, 1e4), (25013, 300, 1e8), (30011, 512, 1e12),
                                       (12007, 512, 1e3)])
def test_wide_factor_against_oracle(cq, orc, m, n, kappa, emulation):
    A = synth.test_matrix(m, n, kappa, rep=31)
    emu = cq.EMU_AUTO if emulation == "auto" else cq.EMU_OFF
    res = cq.factor(cq.to_colmajor(A), opts=cq.default_opts(emulation=emu), check=False)
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
    # the first shift from the Gramian's norm (Alg. 1)
    lam = orc.sym_norm2(orc.gram(A))
    assert res.info["sigma_first"] == pytest.approx(orc.shift(m, n, lam), rel=1e-2)


def partials_max():
    return 2 * torch.cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("emulation", ["auto", "off"])
@pytest.mark.parametrize("m,n", [(30011, 256), (20011, 512), (7001, 449)])
def test_wide_gramian_against_oracle(cq, orc, m, n, emulation):
    A = synth.test_matrix(m, n, 1e8, rep=32)
    emu = cq.EMU_AUTO if emulation == "auto" else cq.EMU_OFF
    X = cq.gram(cq.to_colmajor(A), opts=cq.default_opts(emulation=emu)).cpu().numpy()
    Xo = orc.gram(A)
    absA = np.abs(A)
    err = np.abs(X - Xo)
    # the oracle's own error plus that of X: the FP64 sweep's m u |A|^T|A|
    # (recursive summation), or for the digit products the single rounding
    # of each row group's partial and their fixed-order sum
    oracle_err = (m * U / (1 - m * U)) * (absA.T @ absA)
    own = oracle_err if emulation == "off" else (partials_max() + 12) * U * (absA.T @ absA)
    bound = oracle_err + own + 1e-300
    assert np.all(err <= bound), float(np.max(err / bound))
    assert np.array_equal(X, X.T)


@pytest.mark.parametrize("m,n", [(20011, 512), (5003, 300)])
def test_wide_gramian_exact_on_integers(cq, m, n):
    """Integer entries in [-1024, 1024]: every product and partial sum is an
    integer below 2^53, so the Gramian is exact in any summation order and
    both kernels must return it bit for bit."""
    rng = np.random.default_rng(n)
    A = rng.integers(-1024, 1025, size=(m, n)).astype(np.float64)
    A[:, 7] = 0.0  # a zero column
    A[:, n - 1] *= 2.0 ** -30  # a column on another scale (still exact)
    Ai = A.copy()
    Ai[:, n - 1] *= 2.0 ** 30
    Xi = Ai.astype(np.int64).T @ Ai.astype(np.int64)  # exact integer Gramian
    Xe = Xi.astype(np.float64)
    Xe[:, n - 1] *= 2.0 ** -30
    Xe[n - 1, :] *= 2.0 ** -30
    for emu in (cq.EMU_AUTO, cq.EMU_OFF):
        X = cq.gram(cq.to_colmajor(A), opts=cq.default_opts(emulation=emu)).cpu().numpy()
        assert np.array_equal(X, Xe), (emu, float(np.max(np.abs(X - Xe))))


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


def test_wide_append_to_empty_basis(cq, orc):
    m, p = 20011, 300
    A = synth.test_matrix(m, p, 1e6, rep=35)
    b = cq.Basis(m, p)
    st, info = b.append(cq.to_colmajor(A))
    assert st == cq.OK, info
    Q, R = b.Q().cpu().numpy(), b.R().cpu().numpy()
    b.close()
    check_orth(Q, "wide append to an empty basis")
    assert orc.rrr(A, Q, np.triu(R)) <= 1e-13
    Qn, Bn, Rn, sto, _ = orc.cholqr_update(np.zeros((m, 0)), A, min_iter=2)
    assert sto >= 0
    check_q(float(np.max(np.abs(Q - Qn))), 1e6, m, "wide append to an empty basis")
    check_r(float(np.max(np.abs(R - Rn))), 1e6, Rn, m, "wide append to an empty basis")


@pytest.mark.parametrize("n", [300, 512])
def test_wide_factor_in_place(cq, n):
    """Q == A: the tensor-core solve of a row tile forms its 64-column output
    blocks from the last to the first, so no block reads a column an earlier
    one overwrote; the result equals the out-of-place one bit for bit."""
    m = 9011
    A = synth.test_matrix(m, n, 1e10, rep=36)
    dA = cq.to_colmajor(A)
    ref = cq.factor(dA, check=False)
    res = cq.factor(dA, Q=dA, check=False)
    torch.cuda.synchronize()
    assert ref.status == cq.OK and res.status == cq.OK
    assert torch.equal(res.Q, ref.Q) and torch.equal(res.R, ref.R)
    assert res.Q.data_ptr() == dA.data_ptr()


@pytest.mark.parametrize("n", [160, 320])
def test_wide_breakdown_and_retry(cq, orc, n):
    """The wide control step's Cholesky is shared by the CTAs of a
    cooperative launch: a zero column makes the unshifted first attempt
    fail at its pivot in every CTA, the shift is recomputed and the retry
    succeeds (SHIFT_ON_BREAKDOWN); without shifts the same matrix breaks
    down.  Counters and the result against the oracle."""
    m = 8009
    A = synth.test_matrix(m, n, 1e2, rep=37)
    A[:, n - 70] = 0.0  # the failing pivot lies in the second 64-column panel or later
    dA = cq.to_colmajor(A)
    res = cq.factor(dA, opts=cq.default_opts(shift_policy=cq.SHIFT_ON_BREAKDOWN), check=False)
    torch.cuda.synchronize()
    Qo, Ro, sto, info_o = orc.cholqr(A, shift_policy=orc.SHIFT_ON_BREAKDOWN)
    assert res.status == sto and res.status >= 0, (res.status, sto)
    assert res.info["shifts"] == info_o.shifts >= 1
    assert res.info["chol_attempts"] == info_o.chol_attempts
    Q, R = res.Q.cpu().numpy(), res.R.cpu().numpy()
    assert orc.rrr(A, Q, R) <= 1e-13
    res0 = cq.factor(dA, opts=cq.default_opts(shift_policy=cq.SHIFT_NONE), check=False)
    torch.cuda.synchronize()
    _, _, sto0, _ = orc.cholqr(A, shift_policy=orc.SHIFT_NONE)
    assert res0.status == sto0 == cq.ERR_BREAKDOWN


def test_wide_mixed_against_oracle(cq, orc):
    """CQR_PREC_MIXED above 128 columns: the FP32 first Gramian with its
    shift, then the FP64 passes of the wide path."""
    m, n, kappa = 20011, 300, 1e10
    A = synth.test_matrix(m, n, kappa, rep=38)
    res = cq.factor(cq.to_colmajor(A), opts=cq.default_opts(precision=cq.PREC_MIXED), check=False)
    torch.cuda.synchronize()
    assert res.status == cq.OK, res.info
    Q, R = res.Q.cpu().numpy(), res.R.cpu().numpy()
    check_orth(Q, "wide mixed")
    assert orc.rrr(A, Q, R) <= 1e-13
    Qo, Ro, sto, _ = orc.cholqr(A)
    assert sto == cq.OK
    check_q(float(np.max(np.abs(Q - Qo))), kappa, m, "wide mixed")
    check_r(float(np.max(np.abs(R - Ro))), kappa, Ro, m, "wide mixed")


def test_wide_sharded_two_ranks(cq, orc):
    """Two row shards as host threads with their own streams on one GPU: each
    forms its wide Gramian, the reducer sums them in rank order, and both
    ranks' cooperative control steps run (one after another on the device's
    cooperative stream) to the same R."""
    import threading
    from paper_2507_07788_gb300.sharded import LocalReducerGroup, factor_sharded, split_rows
    m, n, kappa, world = 20011, 200, 1e8, 2
    A = synth.test_matrix(m, n, kappa, rep=39)
    grp = LocalReducerGroup(world, n * n, timeout_s=60.0)
    shards = [cq.to_colmajor(A[r0:r1]) for r0, r1 in split_rows(m, world)]
    torch.cuda.synchronize()
    out = [None] * world

    def rank_main(r):
        torch.cuda.set_device(0)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            out[r] = factor_sharded(shards[r], m, grp.reducer(r), stream=s, check=False)
        s.synchronize()

    th = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for r in range(world):
        assert out[r].status == cq.OK, (r, out[r].status, grp.reducer(r).error)
    assert torch.equal(out[0].R, out[1].R)
    Q = np.vstack([o.Q.cpu().numpy() for o in out])
    R = np.triu(out[0].R.cpu().numpy())
    check_orth(Q, "wide sharded")
    assert orc.rrr(A, Q, R) <= 1e-13
    Qo, Ro, sto, _ = orc.cholqr(A)
    assert sto == cq.OK
    check_q(float(np.max(np.abs(Q - Qo))), kappa, m, "wide sharded")
    check_r(float(np.max(np.abs(R - Ro))), kappa, Ro, m, "wide sharded")


def test_wide_concurrent_streams(cq):
    """Two wide factorisations issued at once from two host threads on two
    streams: their cooperative control steps take turns on the device's
    cooperative stream, and each result equals the same call made alone,
    bit for bit."""
    import threading
    m = 15013
    mats = [cq.to_colmajor(synth.test_matrix(m, n, 1e10, rep=40 + n)) for n in (300, 512)]
    alone = [cq.factor(dA, check=False) for dA in mats]
    torch.cuda.synchronize()
    out = [None, None]

    def run(i):
        torch.cuda.set_device(0)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            out[i] = cq.factor(mats[i], stream=s, check=False)
        s.synchronize()

    th = [threading.Thread(target=run, args=(i,)) for i in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for i in range(2):
        assert alone[i].status == cq.OK and out[i].status == cq.OK, (alone[i].status, out[i].status)
        assert torch.equal(out[i].Q, alone[i].Q) and torch.equal(out[i].R, alone[i].R)
