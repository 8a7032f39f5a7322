"""Serving runtime (cqr_server_*): continuous batching over resident bases.

The same request stream is executed twice on fresh bases: once with every
request submitted only after the previous one completed ("alone"), once with
all requests in flight together ("mix", batched appends and concurrent
workers).  Each basis must end bitwise identical, because a batched problem
runs the same per-CTA work and reduction order as alone.  The result is also
checked against direct library calls, for orthogonality, and against the
oracle: the request stream replayed through the oracle (sCholQR3 for a
factor request, Alg. 2 for an append) gives every basis's Q and R, compared
entry by entry within the bounds of tests/parity.py."""
import numpy as np
import pytest

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


def snapshot(bases):
    return [(b.Q().cpu().numpy().copy(), b.R().cpu().numpy().copy()) for b in bases]


def test_same_alone_and_in_the_mix(cq, orc):
    from paper_2507_07788_gb300 import serve_driver as sd
    wl = sd.make_workload(n_bases=6, n_requests=40, mean_gap_s=1e-4, m_lo=3000, m_hi=120_000,
                          n_lo=4, n_hi=24, p_lo=2, p_hi=12, n_max=96, seed=3)
    sd.make_payloads(wl, seed=3)
    srv = cq.Server(slots=3, batch_max=8, hbm_budget_bytes=1 << 30, small_rows=60_000)
    b1 = sd.make_bases(cq, wl)
    sd.run_alone(cq, srv, b1, wl)
    alone = snapshot(b1)
    res_alone = [r.result for r in wl.reqs]
    b2 = sd.make_bases(cq, wl)
    sd.replay(cq, srv, b2, wl, realtime=False)
    mix = snapshot(b2)
    res_mix = [r.result for r in wl.reqs]
    srv.close()
    assert all(r["status"] >= 0 for r in res_alone), res_alone
    assert all(r["status"] >= 0 for r in res_mix), res_mix
    assert any(r["batch_size"] > 1 for r in res_mix), "no batch formed in the mix"
    for (Qa, Ra), (Qm, Rm) in zip(alone, mix):
        assert np.array_equal(Qa, Qm) and np.array_equal(Ra, Rm)
    for (Qa, _), mb in zip(alone, wl.m):
        if Qa.shape[1]:
            check_orth(Qa, "served basis")
    # the served results against the oracle's replay of the same stream
    ref, statuses = oracle_replay(orc, wl)
    for r, st_o in zip(wl.reqs, statuses):
        assert st_o >= 0, (r.kind, r.result, st_o)
    for bi, ((Qa, Ra), (Qo, Ro)) in enumerate(zip(alone, ref)):
        assert Qa.shape == Qo.shape, bi
        if Qa.shape[1] == 0:
            continue
        q = Qa.shape[1]
        sv = np.linalg.svd(Ro, compute_uv=False)
        kap = sv[0] / sv[-1]
        check_q(float(np.max(np.abs(Qa - Qo))), kap, Qa.shape[0], f"served basis {bi}")
        check_r(float(np.max(np.abs(np.triu(Ra[:q, :q]) - Ro))), kap, Ro, Qa.shape[0], f"served basis {bi}")
    for b in b1 + b2:
        b.close()


def oracle_replay(orc, wl):
    """Each basis's (Q, R) after the request stream, computed by the oracle:
    a factor request replaces the basis by the sCholQR3 factors of its
    payload, an append extends it by Alg. 2 (two outer iterations at least,
    the library's default).  Returns the states and each request's status."""
    statuses = []
    state = [(np.zeros((mb, 0), order="F"), np.zeros((0, 0))) for mb in wl.m]
    for r in wl.reqs:
        A = np.asfortranarray(r.payload.cpu().numpy())
        Q, R = state[r.basis]
        if r.kind == "factor":
            Qn, Rn, st, _ = orc.cholqr(A)
            state[r.basis] = (np.asfortranarray(Qn), np.triu(Rn))
        else:
            Qn, Bn, Rn, st, _ = orc.cholqr_update(Q, A, min_iter=2)
            q, p = Q.shape[1], A.shape[1]
            Rb = np.block([[R, Bn], [np.zeros((p, q)), np.triu(Rn)]])
            state[r.basis] = (np.asfortranarray(np.hstack([Q, Qn])), Rb)
        statuses.append(st)
    return state, statuses


def test_batched_append_matches_direct_call(cq):
    m, p = 20000, 6
    rng = np.random.default_rng(0)
    base = cq.to_colmajor(rng.standard_normal((m, 10)))
    blk = cq.to_colmajor(rng.standard_normal((m, p)))
    direct = cq.Basis(m, 32)
    direct.append(base)
    direct.append(blk)
    srv = cq.Server(slots=1, batch_max=4, small_rows=100_000)
    served = cq.Basis(m, 32)
    r1 = srv.wait(srv.submit_append(served, base))
    r2 = srv.wait(srv.submit_append(served, blk))
    srv.close()
    assert r1["batched"] == 1 and r2["batched"] == 1
    assert np.array_equal(direct.Q().cpu().numpy(), served.Q().cpu().numpy())
    assert np.array_equal(direct.R().cpu().numpy(), served.R().cpu().numpy())
    direct.close()
    served.close()


def test_factor_request_replaces_basis(cq, orc):
    from paper_2507_07788_gb300 import synth
    m, n = 30000, 12
    A = synth.test_matrix(m, n, 1e8, rep=1)
    dA = cq.to_colmajor(A)
    b = cq.Basis(m, 40)
    b.append(cq.to_colmajor(synth.gaussian(m, 20, seed=1)))
    srv = cq.Server(slots=2, batch_max=0)
    r = srv.wait(srv.submit_factor(b, dA))
    srv.close()
    assert r["status"] == cq.OK and r["kind"] == 0 and b.cols == n
    res = cq.factor(dA)
    assert np.array_equal(b.Q().cpu().numpy(), res.Q.cpu().numpy())
    assert np.array_equal(b.R().cpu().numpy(), res.R.cpu().numpy())
    b.close()


def test_hbm_budget_limits_concurrency(cq):
    from paper_2507_07788_gb300 import serve_driver as sd
    wl = sd.make_workload(n_bases=4, n_requests=8, mean_gap_s=1e-5, m_lo=200_000, m_hi=200_001,
                          n_lo=16, n_hi=16, factor_frac=1.0, n_max=32, seed=5)
    sd.make_payloads(wl, seed=5)
    # budget below two factors' staging: admissions are serialised
    srv = cq.Server(slots=4, batch_max=0, hbm_budget_bytes=40 << 20)
    bases = sd.make_bases(cq, wl)
    sd.replay(cq, srv, bases, wl, realtime=False)
    srv.close()
    iv = sorted((r.result["t_start"], r.result["t_done"]) for r in wl.reqs)
    for (s0, d0), (s1, d1) in zip(iv, iv[1:]):
        assert s1 >= d0 - 1e-6, "two requests ran together beyond the budget"
    assert all(r.result["status"] == cq.OK for r in wl.reqs)
    for b in bases:
        b.close()


def test_cached_basis_through_the_server(cq, orc):
    # a basis with a digit cache: the factor request refills the cache for
    # its new columns, and small appends go to basis_append (which keeps the
    # cache) instead of the batched launch; the cached cross Gramian and
    # projection then see the factor's columns, not the ones it replaced
    from paper_2507_07788_gb300 import synth
    m, n, p = 300007, 16, 8
    b = cq.Basis(m, 48)
    b.enable_digit_cache()
    b.append(cq.to_colmajor(synth.gaussian(m, 20, seed=11)))
    A = synth.test_matrix(m, n, 1e8, rep=2)
    srv = cq.Server(slots=2, batch_max=8, small_rows=400_000)
    r = srv.wait(srv.submit_factor(b, cq.to_colmajor(A)))
    assert r["status"] == cq.OK and b.cols == n
    Qf = b.Q().cpu().numpy()[:, :n]
    rng = np.random.default_rng(12)
    blocks = [A]
    for k in range(2):
        blk = Qf @ rng.standard_normal((n, p)) * 0.1 + synth.gaussian(m, p, seed=20 + k) * 1e-3
        blocks.append(blk)
        r = srv.wait(srv.submit_append(b, cq.to_colmajor(blk)))
        assert r["status"] >= 0 and r["batched"] == 0, r
    srv.close()
    q = n + 2 * p
    assert b.cols == q
    Q = b.Q().cpu().numpy()[:, :q]
    R = b.R().cpu().numpy()[:q, :q]
    X = np.hstack(blocks)
    assert orc.loo_frob(Q) <= 1e-12
    assert np.linalg.norm(X - Q @ R) / np.linalg.norm(X) <= 1e-13
    b.close()
