"""Parity of basis_create / basis_append (Alg. 2 on the GPU, through the C ABI)
with the CPU oracle's Alg. 2, append by append, on near-dependent blocks
(block_k = Q_prev G 0.1 + N eta, eta log-uniform in [1e-12, 1]).

Element-wise bounds scale with kappa of the concatenated blocks so far: a
near-dependent block early in the run makes every later factor as sensitive
as that block (QR perturbation theory), whatever the later block looks like.
The bounds are those of the factorisation (tests/parity.py): entries of the
new columns of Q within max(1e-12, 4 kappa u / sqrt(m)), of the new columns
of R within 4 kappa u max(|R|, |B|), and ||[Q_in Q]^T [Q_in Q] - I||_F
<= 1e-13 after every append (the Gramian summed over row blocks)."""
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


def test_basis_growth_matches_oracle(cq, orc):
    m, p, count = 5003, 8, 8
    blocks, etas = synth.basis_growth_blocks(m, p, count, seed=1)
    b = cq.Basis(m, p * count)
    Qo = np.zeros((m, 0))
    Ro = np.zeros((0, 0))
    for k, blk in enumerate(blocks):
        st, info = b.append(cq.to_colmajor(blk))
        Qn, Bn, Rn, sto, info_o = orc.cholqr_update(Qo, blk, min_iter=2)
        assert st == sto and st >= 0, (k, st, info, info_o)
        q = Qo.shape[1]
        Qo = np.hstack([Qo, Qn])
        Ro = np.block([[Ro, Bn], [np.zeros((p, q)), Rn]])
        Qg = b.Q().cpu().numpy()
        Rg = b.R().cpu().numpy()
        assert Qg.shape == (m, q + p)
        # orthogonality after every append
        check_orth(Qg, f"growth append {k}")
        # reconstruction of all blocks so far
        Afull = np.hstack(blocks[: k + 1])
        assert orc.rrr(Afull, Qg, Rg) <= 1e-13, k
        # element-wise parity: the QR factors of [A_prev A_in] are unique and
        # their forward error scales with kappa([A_prev A_in]) (a library SVD
        # of the test input gives it), relative to the size of the factors
        scale = max(np.max(np.abs(Rn)), np.max(np.abs(Bn)) if q else 0.0)
        sv = np.linalg.svd(Afull, compute_uv=False)
        kap = sv[0] / sv[-1]
        dR = np.max(np.abs(Rg[: q + p, q:] - Ro[: q + p, q:]))
        dQ = np.max(np.abs(Qg[:, q:] - Qn))
        print(f"append {k}: eta={etas[k]:.1e} iters={info['iters']}/{info_o.iters} "
              f"shifts={info['shifts']}/{info_o.shifts} dR={dR:.2e} dQ={dQ:.2e}")
        check_r(dR, kap, np.array([scale]), m, f"growth append {k}")
        check_q(dQ, kap, m, f"growth append {k}")
    b.close()


def test_first_append_equals_factor(cq):
    A = synth.test_matrix(4001, 12, 1e6, rep=2)
    b = cq.Basis(4001, 12)
    st, info = b.append(cq.to_colmajor(A))
    res = cq.factor(cq.to_colmajor(A))
    assert st >= 0
    Rb = b.R().cpu().numpy()
    Rf = res.R.cpu().numpy()
    assert np.max(np.abs(Rb - Rf)) <= 1e-10 * np.max(np.abs(Rf))
    b.close()


def test_capacity_error_keeps_basis(cq):
    m = 2000
    b = cq.Basis(m, 10)
    A = synth.gaussian(m, 8, seed=3)
    st, _ = b.append(cq.to_colmajor(A))
    assert st == cq.OK and b.cols == 8
    Q0 = b.Q().cpu().numpy().copy()
    st, _ = b.append(cq.to_colmajor(synth.gaussian(m, 4, seed=4)), check=False)
    assert st == cq.ERR_CAPACITY and b.cols == 8
    assert np.array_equal(b.Q().cpu().numpy(), Q0)
    b.close()


def test_dependent_column_lucky_breakdown(cq, orc):
    m, q, p = 3000, 6, 4
    b = cq.Basis(m, 16)
    base = synth.gaussian(m, q, seed=5)
    b.append(cq.to_colmajor(base))
    Qin = b.Q().cpu().numpy()
    A = synth.gaussian(m, p, seed=6)
    A[:, 2] = Qin @ np.array([1.0, -2.0, 0.5, 0.0, 3.0, 1.0])
    st, info = b.append(cq.to_colmajor(A))
    assert st >= 0 and info["shifts"] >= 1
    Qg = b.Q().cpu().numpy()
    check_orth(Qg, "lucky breakdown")


def test_breakdown_leaves_basis_unchanged(cq):
    m = 1500
    b = cq.Basis(m, 16, opts=cq.default_opts(max_escalations=0))
    b.append(cq.to_colmajor(synth.gaussian(m, 4, seed=7)))
    Q0, R0 = b.Q().cpu().numpy().copy(), b.R().cpu().numpy().copy()
    bad = synth.gaussian(m, 4, seed=8)
    bad[5, 1] = np.nan
    st, info = b.append(cq.to_colmajor(bad), check=False)
    assert st == cq.ERR_BREAKDOWN
    assert b.cols == 4
    assert np.array_equal(b.Q().cpu().numpy(), Q0) and np.array_equal(b.R().cpu().numpy(), R0)
    b.close()


def test_wide_basis_split_sweep(cq, orc):
    # q p + p (p+1)/2 beyond one CTA's entry budget: the solve and the Gram
    # sweep run as two kernels
    m, p = 2500, 32
    b = cq.Basis(m, 320)
    for k in range(9):
        st, info = b.append(cq.to_colmajor(synth.gaussian(m, p, seed=20 + k)))
        assert st >= 0
    Qg = b.Q().cpu().numpy()
    assert Qg.shape[1] == 288
    check_orth(Qg, "wide basis split sweep")
    b.close()


def _check_append(orc, Qo, Ro, blk, Qg, Rg, m, info, k):
    """One append against the oracle's Alg. 2 (as in the growth test)."""
    p = blk.shape[1]
    Qn, Bn, Rn, sto, info_o = orc.cholqr_update(Qo, blk, min_iter=2)
    q = Qo.shape[1]
    Qo2 = np.hstack([Qo, Qn])
    Ro2 = np.block([[Ro, Bn], [np.zeros((p, q)), Rn]])
    assert Qg.shape == (m, q + p)
    check_orth(Qg, f"append {k} p={p} (m={m})")
    scale = max(np.max(np.abs(Rn)), np.max(np.abs(Bn)) if q else 0.0)
    dR = np.max(np.abs(Rg[: q + p, q:] - Ro2[: q + p, q:]))
    dQ = np.max(np.abs(Qg[:, q:] - Qn))
    return Qo2, Ro2, dR, dQ, scale, sto, info_o


@pytest.mark.parametrize("widths", [(32, 40), (64, 8, 32), (8, 20)])
def test_tall_basis_tensor_cross_gramian(cq, orc, widths):
    # m above the row limit of the serving runtime's batched appends: appends
    # of 32..64 columns form the cross Gramian [Q_in Y]^T Y of every iteration
    # on the tensor cores (p = 32: 32-wide kernel; 40, 64: 64-wide), narrower
    # ones keep the fused FP64 sweep; both must follow the oracle
    m = 300007
    b = cq.Basis(m, sum(widths))
    Qo = np.zeros((m, 0))
    Ro = np.zeros((0, 0))
    blocks = []
    rng = np.random.default_rng(77)
    for k, p in enumerate(widths):
        if k == 0:
            blk = synth.gaussian(m, p, seed=70 + k)
        else:
            # near-dependent on the basis so far (the growth recipe)
            blk = Qo @ rng.standard_normal((Qo.shape[1], p)) * 0.1 + synth.gaussian(m, p, seed=70 + k) * 1e-6
        blocks.append(blk)
        st, info = b.append(cq.to_colmajor(blk))
        Qg, Rg = b.Q().cpu().numpy(), b.R().cpu().numpy()
        Qo, Ro, dR, dQ, scale, sto, info_o = _check_append(orc, Qo, Ro, blk, Qg, Rg, m, info, k)
        assert st == sto and st >= 0, (k, st, info, info_o)
        Afull = np.hstack(blocks)
        assert orc.rrr(Afull, Qg, Rg) <= 1e-13, k
        sv = np.linalg.svd(Afull, compute_uv=False)
        kap = sv[0] / sv[-1]
        q = Qg.shape[1] - p
        print(f"append {k} p={p}: iters={info['iters']}/{info_o.iters} dR={dR:.2e} dQ={dQ:.2e} kappa={kap:.1e}")
        check_r(dR, kap, np.array([scale]), m, f"append {k} p={p} q={q} (m={m})")
        check_q(dQ, kap, m, f"append {k} p={p} q={q} (m={m})")
    b.close()


def test_tall_basis_nan_breaks_down(cq):
    m = 300007
    b = cq.Basis(m, 16, opts=cq.default_opts(max_escalations=0))
    b.append(cq.to_colmajor(synth.gaussian(m, 8, seed=80)))
    bad = synth.gaussian(m, 8, seed=81)
    bad[123456, 3] = np.nan
    st, info = b.append(cq.to_colmajor(bad), check=False)
    assert st == cq.ERR_BREAKDOWN and b.cols == 8
    b.close()


@pytest.mark.parametrize("widths", [(8, 8, 16, 4, 8), (64, 8, 1)])
def test_tall_basis_digit_cache(cq, orc, widths):
    # a basis that keeps the digits of its columns: appends of <= 16 columns
    # form their cross Gramian from the cached digits of Q_in on the tensor
    # cores (the first append, to the empty basis, takes the factorisation's
    # pipeline; wide ones the split cross Gramian); all follow the oracle
    m = 300007
    b = cq.Basis(m, sum(widths))
    b.enable_digit_cache()
    Qo = np.zeros((m, 0))
    Ro = np.zeros((0, 0))
    blocks = []
    rng = np.random.default_rng(91)
    for k, p in enumerate(widths):
        if k == 0:
            blk = synth.gaussian(m, p, seed=90 + k)
        else:
            blk = Qo @ rng.standard_normal((Qo.shape[1], p)) * 0.1 + synth.gaussian(m, p, seed=90 + k) * 1e-6
        blocks.append(blk)
        st, info = b.append(cq.to_colmajor(blk))
        Qg, Rg = b.Q().cpu().numpy(), b.R().cpu().numpy()
        Qo, Ro, dR, dQ, scale, sto, info_o = _check_append(orc, Qo, Ro, blk, Qg, Rg, m, info, k)
        assert st == sto and st >= 0, (k, st, info, info_o)
        Afull = np.hstack(blocks)
        assert orc.rrr(Afull, Qg, Rg) <= 1e-13, k
        sv = np.linalg.svd(Afull, compute_uv=False)
        kap = sv[0] / sv[-1]
        q = Qg.shape[1] - p
        print(f"append {k} p={p}: iters={info['iters']}/{info_o.iters} dR={dR:.2e} dQ={dQ:.2e} kappa={kap:.1e}")
        check_r(dR, kap, np.array([scale]), m, f"append {k} p={p} q={q} (m={m})")
        check_q(dQ, kap, m, f"append {k} p={p} q={q} (m={m})")
    b.close()


def test_digit_cache_enabled_late_and_nan(cq, orc):
    # the cache filled for columns already in the basis, then a NaN append
    # breaks down and leaves basis and cache in use for the next append
    m = 300007
    b = cq.Basis(m, 24, opts=cq.default_opts(max_escalations=0))
    b.append(cq.to_colmajor(synth.gaussian(m, 8, seed=95)))
    b.enable_digit_cache()
    b.enable_digit_cache()  # a second call is a no-op
    bad = synth.gaussian(m, 8, seed=96)
    bad[123456, 3] = np.nan
    st, info = b.append(cq.to_colmajor(bad), check=False)
    assert st == cq.ERR_BREAKDOWN and b.cols == 8
    nxt = synth.gaussian(m, 8, seed=97)
    st, info = b.append(cq.to_colmajor(nxt))
    assert st == cq.OK and b.cols == 16
    Qg = b.Q().cpu().numpy()
    check_orth(Qg, "cache enabled late")
    b.close()


def test_digit_cache_beyond_projection_width(cq, orc):
    # q > 256: the narrow append keeps the FP64 projection and solve, its cross
    # Gramian still reads the cached digits (five 64-column Z blocks)
    m = 300007
    widths = (128, 128, 8, 8)
    b = cq.Basis(m, sum(widths))
    b.enable_digit_cache()
    Qo = np.zeros((m, 0))
    Ro = np.zeros((0, 0))
    rng = np.random.default_rng(93)
    blocks = []
    for k, p in enumerate(widths):
        if k == 0:
            blk = synth.gaussian(m, p, seed=100 + k)
        else:
            blk = Qo @ rng.standard_normal((Qo.shape[1], p)) * 0.1 + synth.gaussian(m, p, seed=100 + k) * 1e-3
        blocks.append(blk)
        st, info = b.append(cq.to_colmajor(blk))
        Qg, Rg = b.Q().cpu().numpy(), b.R().cpu().numpy()
        Qo, Ro, dR, dQ, scale, sto, info_o = _check_append(orc, Qo, Ro, blk, Qg, Rg, m, info, k)
        assert st == sto and st >= 0, (k, st, info, info_o)
        Afull = np.hstack(blocks)
        assert orc.rrr(Afull, Qg, Rg) <= 1e-13, k
        sv = np.linalg.svd(Afull, compute_uv=False)
        kap = sv[0] / sv[-1]
        q = Qg.shape[1] - p
        print(f"append {k} p={p}: iters={info['iters']}/{info_o.iters} dR={dR:.2e} dQ={dQ:.2e} kappa={kap:.1e}")
        check_r(dR, kap, np.array([scale]), m, f"beyond projection width append {k}")
        check_q(dQ, kap, m, f"beyond projection width append {k}")
    b.close()
