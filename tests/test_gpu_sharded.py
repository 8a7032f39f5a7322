"""Row-sharded sCholQR3 (cholqr_factor_sharded) with simulated ranks on one
GPU: each rank is a host thread with its own stream and row shard, and the
ranks exchange their Gramian partials through LocalReducerGroup (host
staging and a barrier).  No kernel waits for another rank: every wait is on
the host, after the rank's own stream has drained.

Checks: the stacked shards of Q and the common R against cholqr_factor of the
whole matrix and against the oracle (bounds of tests/parity.py); R bitwise
the same on every rank; one rank equal to cholqr_factor bit for bit; and a
rank whose peer never joins gets CQR_ERR_REDUCE after the reducer's timeout,
with the GPU still usable afterwards.
"""
import threading

import numpy as np
import pytest

from paper_2507_07788_gb300 import synth
from parity import check_orth, check_q, check_r

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


def run_sharded(cq, A, world, opts=None, timeout_s=60.0):
    from paper_2507_07788_gb300.sharded import LocalReducerGroup, factor_sharded, split_rows
    m, n = A.shape
    grp = LocalReducerGroup(world, n * n, timeout_s=timeout_s)
    blocks = split_rows(m, world)
    shards = [cq.to_colmajor(A[r0:r1]) for r0, r1 in blocks]
    torch.cuda.synchronize()
    out = [None] * world

    def rank_main(r):
        torch.cuda.set_device(0)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            out[r] = factor_sharded(shards[r], m, grp.reducer(r), opts=opts, stream=s, check=False)
        s.synchronize()

    th = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    return out, grp


@pytest.mark.parametrize("world,m,n,kappa", [(2, 40013, 64, 1e12), (3, 20011, 20, 1e8),
                                              (2, 400003, 48, 1e10)])
def test_sharded_matches_factor_and_oracle(cq, orc, world, m, n, kappa):
    A = synth.test_matrix(m, n, kappa, rep=17)
    out, grp = run_sharded(cq, A, world)
    for r in range(world):
        assert out[r].status == cq.OK, (r, out[r].status, grp.reducer(r).error)
        assert out[r].info == out[0].info
    Rs = [o.R.cpu().numpy() for o in out]
    for R in Rs[1:]:
        assert np.array_equal(R, Rs[0])  # the same decisions and R on every rank
    Q = np.vstack([o.Q.cpu().numpy() for o in out])
    R = np.triu(Rs[0])
    check_orth(Q, f"sharded world={world} {m}x{n}")
    assert orc.rrr(A, Q, R) <= 1e-13
    full = cq.factor(cq.to_colmajor(A))
    torch.cuda.synchronize()
    check_q(np.max(np.abs(Q - full.Q.cpu().numpy())), kappa, m, f"sharded vs factor world={world}")
    check_r(np.max(np.abs(R - full.R.cpu().numpy())), kappa, full.R.cpu().numpy(), m,
            f"sharded vs factor world={world}")
    Qo, Ro, sto, info_o = orc.cholqr(A)
    assert sto == cq.OK
    check_q(np.max(np.abs(Q - Qo)), kappa, m, f"sharded vs oracle world={world}")
    check_r(np.max(np.abs(R - Ro)), kappa, Ro, m, f"sharded vs oracle world={world}")


def test_one_rank_is_cholqr_factor(cq):
    A = synth.test_matrix(30011, 40, 1e10, rep=18)
    out, _ = run_sharded(cq, A, 1)
    full = cq.factor(cq.to_colmajor(A))
    torch.cuda.synchronize()
    assert out[0].status == full.status == cq.OK
    assert out[0].info == full.info
    assert torch.equal(out[0].Q, full.Q) and torch.equal(out[0].R, full.R)


def test_absent_peer_reports_reduce_failure(cq):
    from paper_2507_07788_gb300.sharded import LocalReducerGroup, factor_sharded
    m, n = 20000, 16
    A = synth.test_matrix(m, n, 1e6, rep=19)
    grp = LocalReducerGroup(2, n * n, timeout_s=1.0)
    dA = cq.to_colmajor(A[: m // 2])
    res = factor_sharded(dA, m, grp.reducer(0), check=False)  # rank 1 never calls
    assert res.status == cq.ERR_REDUCE
    assert grp.reducer(0).error is not None
    # the context is still usable
    ok = cq.factor(cq.to_colmajor(A))
    assert ok.status == cq.OK


def test_sharded_argument_checks(cq):
    from paper_2507_07788_gb300.sharded import LocalReducerGroup, factor_sharded
    A = cq.to_colmajor(synth.test_matrix(1000, 8, 10.0))
    grp = LocalReducerGroup(2, 8 * 8)
    # m_total below the shard's rows, and a reducer too small for n * n
    assert factor_sharded(A, 999, grp.reducer(0), check=False).status == cq.ERR_INVALID
    small = LocalReducerGroup(2, 16)
    assert factor_sharded(A, 2000, small.reducer(0), check=False).status == cq.ERR_INVALID
