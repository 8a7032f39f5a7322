"""Parity of cholqr_factor (CUDA, through the C ABI) with the CPU oracle.

Tolerances (tests/parity.py).  The QR factors of a full-rank A are unique
(positive diagonal of R), but two backward-stable computations that round
differently agree only up to the conditioning of the QR factors: the factors
differ by O(kappa(A) u), and Q's entries are O(1/sqrt(m)).  The tests bound
  |Q_gpu - Q_oracle|_max <= max(1e-12, 4 kappa u / sqrt(m)),
  |R_gpu - R_oracle|_max <= 4 kappa u ||R||_max (+ u ||R||_max),
and require the orthogonality ||Q^T Q - I||_F <= 1e-13 and the residual
||A - QR||_F/||A||_F <= 1e-13 for kappa <= 1e15 outright.  For
kappa <= 1e4 the elementwise Q bound is the 1e-12 the target states.
"""
import math

import numpy as np
import pytest

from paper_2507_07788_gb300 import synth
from parity import U, check_q, check_r, q_tol, r_tol

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


def loo_blocked(Q, rows=2048):
    # ||Q^T Q - I||_F with the Gramian summed over row blocks of 2048: the
    # oracle's row-by-row sum carries a rounding error near u sqrt(m/3) on
    # each diagonal entry (3e-14 at m = 2e5), the size of the 1e-13 bound
    # itself at n = 100; blocking cuts it to u (sqrt(rows) + m / rows)
    m, n = Q.shape
    G = np.zeros((n, n))
    for r0 in range(0, m, rows):
        B = Q[r0:r0 + rows]
        G += B.T @ B
    return float(np.linalg.norm(G - np.eye(n)))


def run_gpu(cq, A, opts=None, inplace=False):
    dA = cq.to_colmajor(A)
    if inplace:
        res = cq.factor(dA, Q=dA, opts=opts, check=False)
    else:
        res = cq.factor(dA, opts=opts, check=False)
    torch.cuda.synchronize()
    return res.Q.cpu().numpy(), res.R.cpu().numpy(), res.status, res.info


@pytest.mark.parametrize("kappa", [1.0, 1e2, 1e4, 1e8, 1e12, 1e15])
@pytest.mark.parametrize("rep", [0, 1])
def test_factor_parity_config1(cq, orc, kappa, rep):
    m, n = 20037, 20  # several tiles, ragged tail
    A = synth.test_matrix(m, n, kappa, rep=rep)
    Q, R, st, info = run_gpu(cq, A)
    Qo, Ro, sto, info_o = orc.cholqr(A)
    assert st == sto == cq.OK, (st, info)
    assert info["iters"] == info_o.iters
    assert info["shifts"] == info_o.shifts
    # shift from the norm estimate: within the paper's eigsh tolerance 1e-2
    assert info["sigma_first"] == pytest.approx(info_o.sigma_first, rel=1e-2)
    assert orc.loo_frob(Q) <= 1e-13
    assert orc.rrr(A, Q, R) <= 1e-13
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    dq = np.max(np.abs(Q - Qo))
    dr = np.max(np.abs(R - Ro))
    print(f"kappa={kappa:.0e} rep={rep} iters={info['iters']} maxdQ={dq:.2e} maxdR={dr:.2e} "
          f"loo={orc.loo_frob(Q):.2e}")
    check_r(dr, kappa, Ro, m, f"config1 kappa={kappa:g} rep={rep}")
    check_q(dq, kappa, m, f"config1 kappa={kappa:g} rep={rep}")


@pytest.mark.parametrize("m,n", [(1, 1), (7, 1), (5, 5), (129, 7), (4000, 16), (3001, 32),
                                 (2500, 64), (1100, 128), (777, 33)])
def test_factor_shapes(cq, orc, m, n):
    A = synth.test_matrix(m, n, 1e3, rep=3)
    Q, R, st, info = run_gpu(cq, A)
    Qo, Ro, sto, info_o = orc.cholqr(A)
    assert st == sto and st >= 0
    assert info["iters"] == info_o.iters
    check_r(np.max(np.abs(R - Ro)), 1e3, Ro, m, f"shape {m}x{n}")
    check_q(np.max(np.abs(Q - Qo)), 1e3, m, f"shape {m}x{n}")


def test_factor_n1_closed_form(cq):
    a = np.random.default_rng(5).standard_normal((10001, 1))
    Q, R, st, info = run_gpu(cq, a)
    nrm = math.sqrt(float(np.sum(a * a)))
    assert st == cq.OK
    assert R[0, 0] == pytest.approx(nrm, rel=1e-13)
    assert np.allclose(Q[:, 0], a[:, 0] / nrm, rtol=0, atol=1e-15)


def test_orthonormal_input_untouched(cq):
    A = np.zeros((4096, 8))
    A[np.arange(8) * 17, np.arange(8)] = 1.0
    Q, R, st, info = run_gpu(cq, A)
    assert st == cq.OK and info["iters"] == 0
    assert np.array_equal(Q, A) and np.array_equal(R, np.eye(8))


def test_in_place(cq, orc):
    A = synth.test_matrix(9999, 24, 1e6, rep=4)
    Q, R, st, info = run_gpu(cq, A, inplace=True)
    Qo, Ro, sto, _ = orc.cholqr(A)
    assert st == cq.OK
    check_q(np.max(np.abs(Q - Qo)), 1e6, 9999, "in place")


def test_leading_dimension(cq, orc):
    m, n, lda = 3000, 10, 3017
    A = synth.test_matrix(m, n, 1e5, rep=5)
    big = cq.colmajor(lda, n)
    big.zero_()
    big[:m].copy_(torch.from_numpy(A))
    dA = big[:m]
    assert dA.stride() == (1, lda)
    res = cq.factor(dA)
    Qo, Ro, _, _ = orc.cholqr(A)
    check_q(np.max(np.abs(res.Q.cpu().numpy() - Qo)), 1e5, m, "leading dimension")


def test_zero_column_forces_shift(cq, orc):
    A = synth.test_matrix(2000, 6, 1e2, rep=6)
    A[:, 3] = 0.0
    opts = cq.default_opts(shift_policy=cq.SHIFT_ON_BREAKDOWN)
    Q, R, st, info = run_gpu(cq, A, opts=opts)
    Qo, Ro, sto, info_o = orc.cholqr(A, shift_policy=orc.SHIFT_ON_BREAKDOWN)
    assert info["shifts"] >= 1 and info_o.shifts >= 1
    assert st >= 0 and sto >= 0
    assert orc.rrr(A, Q, R) <= 1e-13


def test_no_shift_policy_breaks_down(cq):
    A = synth.test_matrix(5000, 12, 1e12)
    opts = cq.default_opts(shift_policy=cq.SHIFT_NONE)
    _, _, st, info = run_gpu(cq, A, opts=opts)
    assert st == cq.ERR_BREAKDOWN


def test_nan_input_reports_breakdown(cq, orc):
    A = synth.test_matrix(1000, 5, 10.0)
    A[17, 2] = np.nan
    _, _, st, info = run_gpu(cq, A)
    _, _, sto, _ = orc.cholqr(A)
    assert st == sto == cq.ERR_BREAKDOWN
    assert info["escalations"] <= cq.default_opts().max_escalations


def test_max_iter_not_converged(cq, orc):
    A = synth.test_matrix(3000, 8, 1e12)
    opts = cq.default_opts(max_iter=1)
    Q, R, st, info = run_gpu(cq, A, opts=opts)
    assert st == cq.NOT_CONVERGED and info["iters"] == 1
    assert orc.rrr(A, Q, R) <= 1e-13


def test_u_sqrt_n_stop_rule(cq, orc):
    A = synth.test_matrix(3000, 8, 1e3)
    opts = cq.default_opts(stop_rule=cq.STOP_U_SQRT_N, max_iter=4)
    _, _, st, info = run_gpu(cq, A, opts=opts)
    _, _, sto, info_o = orc.cholqr(A, stop_rule=orc.STOP_U_SQRT_N, max_iter=4)
    assert st in (cq.OK, cq.NOT_CONVERGED)
    assert info["iters"] <= 4


def test_kappa_1e20_rscholqr(cq, orc):
    # beyond 1/u: the recomputed shift still gives an orthonormal Q (Fig. 1)
    A = synth.test_matrix(20000, 20, 1e20, rep=2)
    Q, R, st, info = run_gpu(cq, A)
    assert st == cq.OK
    assert orc.loo(Q) < 3.16e-13
    assert orc.rrr(A, Q, R) <= 1e-13


@pytest.mark.parametrize("n", [20, 64, 128])
@pytest.mark.parametrize("kappa", [1e8, 1e15, 1e20])
def test_factor_on_the_papers_scale(cq, orc, n, kappa):
    # singular values from 1 up to kappa, as Sec. 4.1 builds them: Gramians
    # of norm up to 1e40, beyond the FP32 range of the norm estimate's power
    # iteration (which runs on X scaled by a power of two); the digit
    # Gramian and solve track FP64 exponents and need no scaling
    m = 20037
    A = synth.test_matrix(m, n, kappa, rep=5, paper_scale=True)
    Q, R, st, info = run_gpu(cq, A)
    assert st == cq.OK, info
    assert orc.loo(Q) < 3.16e-13 and orc.loo_frob(Q) <= 1e-13
    assert orc.rrr(A, Q, R) <= 1e-13
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    X = orc.gram(A)
    assert info["sigma_first"] == pytest.approx(orc.shift(m, n, orc.sym_norm2(X)), rel=1e-2)
    if kappa <= 1e15:
        Qo, Ro, sto, info_o = orc.cholqr(A)
        assert sto == cq.OK and abs(info["iters"] - info_o.iters) <= 1
        check_r(np.max(np.abs(R - Ro)), kappa, Ro, m, f"paper scale n={n} kappa={kappa:g}")
        check_q(np.max(np.abs(Q - Qo)), kappa, m, f"paper scale n={n} kappa={kappa:g}")


def test_deterministic(cq):
    A = synth.test_matrix(50000, 32, 1e10, rep=8)
    Q1, R1, _, _ = run_gpu(cq, A)
    Q2, R2, _, _ = run_gpu(cq, A)
    assert np.array_equal(Q1, Q2) and np.array_equal(R1, R2)


@pytest.mark.parametrize("m,n,kappa,q_kind", [
    (12345, 16, 1e8, "pinned"),      # one row chunk
    (200003, 48, 1e12, "pinned"),    # two row chunks, tensor-core solve, ragged tail
    (200003, 16, 1.0, "pinned"),     # converges before the pre-launched passes end
    (200003, 48, 1e4, "pageable"),   # Q not device-addressable: one copy at the end
    (170001, 40, 1e10, "strided"),   # ldq > m, lda > m
    (200003, 100, 1e12, "pinned"),   # n > 64: the 128-wide digit solve, half-height chunks
])
def test_host_entry_point(cq, orc, m, n, kappa, q_kind):
    # cholqr_factor_host copies A in, factors it exactly as cholqr_factor
    # does and, with a pinned Q, writes the last pass's row chunks to the
    # host as they are solved: the result is bit for bit the device one
    A = synth.test_matrix(m, n, kappa, rep=9)
    Ah = torch.from_numpy(np.asfortranarray(A)).t()
    lda_pad = 5 if q_kind == "strided" else 0
    Abig = torch.zeros((n, m + lda_pad), dtype=torch.float64)
    Abig[:, :m] = Ah
    Ah = Abig.t()[:m]
    if q_kind == "pinned":
        Q = torch.full((n, m), np.nan, dtype=torch.float64, pin_memory=True).t()
    elif q_kind == "pageable":
        Q = torch.full((n, m), np.nan, dtype=torch.float64).t()
    else:
        Q = torch.full((n, m + 7), np.nan, dtype=torch.float64, pin_memory=True).t()[:m]
    res = cq.factor_host(Ah, Q=Q)
    Qh, Rh = res.Q.numpy(), res.R.numpy()
    Qd, Rd, std, infod = run_gpu(cq, A)
    assert res.status == std == cq.OK
    assert res.info == infod
    assert np.array_equal(Qh, Qd) and np.array_equal(Rh, Rd)
    assert loo_blocked(Qh) <= 1e-13
    assert orc.rrr(A, Qh, Rh) <= 1e-13
    assert np.array_equal(Ah.numpy(), A)  # input untouched
    if q_kind == "strided":
        assert torch.isnan(Q.as_strided((7, n), (1, m + 7), m)).all()  # padding untouched


def test_host_entry_point_last_pass_not_foreseen(cq):
    # orthogonal columns of norms 1..2 with no shift: one pass is the last,
    # although its input was far from orthonormal (||Q^T Q - I||_F = 11),
    # so no Q chunk reaches the host during it and every chunk is copied
    # after the stop
    m, n = 200003, 48
    A = synth.orthonormal(m, n, 3) * np.linspace(1.0, 2.0, n)
    opts = cq.default_opts(shift_policy=cq.SHIFT_NONE)
    Q = torch.full((n, m), np.nan, dtype=torch.float64, pin_memory=True).t()
    res = cq.factor_host(A, Q=Q, opts=opts)
    Qd, Rd, std, infod = run_gpu(cq, A, opts=opts)
    assert res.status == std == cq.OK and res.info["iters"] == infod["iters"] == 1
    assert loo_blocked(res.Q.numpy()) <= 1e-13
    assert np.array_equal(res.Q.numpy(), Qd) and np.array_equal(res.R.numpy(), Rd)


def test_host_entry_point_orthonormal_input(cq):
    # X = I on the first Gramian: no pass runs and Q = A, R = I (Alg. 1)
    m, n = 160003, 8
    A = np.zeros((m, n))
    A[np.arange(n) * 1000, np.arange(n)] = 1.0
    Q = torch.full((n, m), np.nan, dtype=torch.float64, pin_memory=True).t()
    res = cq.factor_host(A, Q=Q)
    assert res.status == cq.OK and res.info["iters"] == 0
    assert np.array_equal(res.Q.numpy(), A)
    assert np.array_equal(res.R.numpy(), np.eye(n))


# ---- tensor-core (Ozaki digit) Gramian vs FP64 CUDA-core Gramian

@pytest.mark.parametrize("kappa", [1e4, 1e12])
@pytest.mark.parametrize("n", [1, 16, 17, 20, 25, 32, 33, 48, 64, 65, 100, 128])
def test_emulated_and_native_gramian_agree(cq, orc, kappa, n):
    m = 30011
    A = synth.test_matrix(m, n, kappa, rep=12)
    Qe, Re, ste, infoe = run_gpu(cq, A)
    Qn, Rn, stn, infon = run_gpu(cq, A, opts=cq.default_opts(emulation=cq.EMU_OFF))
    Qo, Ro, sto, info_o = orc.cholqr(A)
    assert ste == stn == sto == cq.OK
    # An unshifted pass whose Gramian sits at the Cholesky breakdown threshold
    # may break down (and take a recomputed shift, then one more pass) on one
    # side only: pass counts may then differ by one, with the shift counts
    # differing too.  Otherwise they agree.
    its = (infoe["iters"], infon["iters"], info_o.iters)
    shs = (infoe["shifts"], infon["shifts"], info_o.shifts)
    assert max(its) - min(its) <= 1
    assert len(set(its)) == 1 or len(set(shs)) > 1, (its, shs)
    for name, Q, R in (("digit", Qe, Re), ("fp64", Qn, Rn)):
        assert orc.loo_frob(Q) <= 1e-13
        assert orc.rrr(A, Q, R) <= 1e-13
        check_r(np.max(np.abs(R - Ro)), kappa, Ro, m, f"{name} n={n} kappa={kappa:g}")
        check_q(np.max(np.abs(Q - Qo)), kappa, m, f"{name} n={n} kappa={kappa:g}")


@pytest.mark.parametrize("n", [64, 100])
def test_chunked_pipeline_parity(cq, orc, n):
    # m large enough that each pass runs as several row chunks (solve of
    # chunk c beside the Gramian of chunk c-1, partials accumulated across
    # chunks): 2 chunks at n = 64, 4 at n = 100, with a ragged last chunk
    m = 160003
    A = synth.test_matrix(m, n, 1e10, rep=15)
    Q, R, st, info = run_gpu(cq, A)
    Qo, Ro, sto, info_o = orc.cholqr(A)
    assert st == sto == cq.OK
    # at this size ||Q^T Q - I||_F after the third pass lies near the 1e-13
    # stop tolerance, so the two sides may stop one pass apart
    assert abs(info["iters"] - info_o.iters) <= 1
    assert orc.loo_frob(Q) <= 1e-13
    assert orc.rrr(A, Q, R) <= 1e-13
    check_r(np.max(np.abs(R - Ro)), 1e10, Ro, m, f"chunked n={n}")
    check_q(np.max(np.abs(Q - Qo)), 1e10, m, f"chunked n={n}")


@pytest.mark.parametrize("n", [8, 24, 48, 100])
def test_emulated_gramian_column_scaling(cq, orc, n):
    # columns scaled over 12 orders of magnitude: each column has its own
    # exponent in the digit Gramian, and the tensor-core solve (n >= 17)
    # balances the columns of Y and the rows of T before splitting them; the
    # result follows the oracle within the bounds of the scaled matrix's
    # condition number
    m = 20000
    A = synth.test_matrix(m, n, 1e3, rep=13)
    As = A * np.resize(np.array([1.0, 1e-6, 1e6, 1e-3, 1e3, 3.0, 1e-5, 1e5]), n)
    kap = np.linalg.cond(As)
    Q, R, st, info = run_gpu(cq, As)
    Qo, Ro, sto, info_o = orc.cholqr(As)
    assert st == sto == cq.OK
    assert orc.loo_frob(Q) <= 1e-13
    assert orc.rrr(As, Q, R) <= 1e-13
    check_q(np.max(np.abs(Q - Qo)), kap, m, f"column scaling n={n}")


@pytest.mark.parametrize("n", [12, 24, 40, 120])
def test_emulated_gramian_row_dynamic_range(cq, orc, n):
    # entries spanning 8 orders of magnitude inside each column
    m = 9000
    rng = np.random.default_rng(14)
    A = rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-4, 4, size=(m, 1))
    kap = np.linalg.cond(A)
    Q, R, st, info = run_gpu(cq, A)
    Qn, Rn, stn, _ = run_gpu(cq, A, opts=cq.default_opts(emulation=cq.EMU_OFF))
    Qo, Ro, sto, _ = orc.cholqr(A)
    assert st == stn == sto == cq.OK
    assert orc.loo_frob(Q) <= 1e-13
    assert orc.rrr(A, Q, R) <= 1e-13
    check_q(np.max(np.abs(Q - Qo)), kap, m, f"row range n={n}")


@pytest.mark.parametrize("m,n", [(130, 17), (5003, 33), (20037, 48), (200003, 64), (257, 64), (129, 20)])
def test_tcgen05_and_mma_sync_paths_agree(cq, orc, m, n):
    # the tcgen05 Gramian and solve (emulation TCGEN05, 17 <= n <= 64) and the
    # default mma.sync digit kernels against each other and the oracle: one
    # tile, a ragged tile of 128 rows, several CTAs
    kappa = 1e8
    A = synth.test_matrix(m, n, kappa, rep=21)
    Qt, Rt, stt, it = run_gpu(cq, A, opts=cq.default_opts(emulation=cq.EMU_TCGEN05))
    Ql, Rl, stl, il = run_gpu(cq, A)
    Qo, Ro, sto, io = orc.cholqr(A)
    assert stt == stl == sto == cq.OK
    assert abs(it["iters"] - il["iters"]) <= 1
    for name, Q, R in (("tcgen05", Qt, Rt), ("mma.sync", Ql, Rl)):
        assert orc.loo_frob(Q) <= 1e-13
        assert orc.rrr(A, Q, R) <= 1e-13
        check_q(np.max(np.abs(Q - Qo)), kappa, m, f"{name} vs oracle {m}x{n}")
        check_r(np.max(np.abs(R - Ro)), kappa, Ro, m, f"{name} vs oracle {m}x{n}")
    check_q(np.max(np.abs(Qt - Ql)), kappa, m, f"tcgen05 vs mma.sync {m}x{n}")
