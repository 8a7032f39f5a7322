"""Basis growth shaped like the basis-growth workload, against the oracle's
Alg. 2 append by append: 32 appends of 8 columns up to n = 256 on 262 147
rows (above the serving runtime's batched-append rows, so every append after
the first reads the basis's digit cache: cross Gramian and, up to q = 256,
projection on the tensor cores).  Block k = Q_prev G 0.1 + N eta with eta
log-uniform in [1e-12, 1] (the first block is N); Q_prev is the oracle's
basis of the blocks so far (a data generator here: an orthonormal basis of
the previous blocks).

After every append: ||[Q_in Q]^T [Q_in Q] - I||_F <= 1e-13 (the Gramian of
the whole basis, updated by the new block's rows and columns), the new
block's residual A_in - [Q_in Q] R[:, q:q+p] <= 1e-13 relative, and the new
columns of Q and R entry by entry against the oracle's within the bounds of
tests/parity.py, with kappa of the concatenated blocks taken from the
oracle's R (the singular values of [A_prev A_in] are those of R).
It runs after the other GPU modules: about a minute of oracle time."""
import numpy as np
import pytest

from paper_2507_07788_gb300 import synth
from parity import ORTH_GATE, check_q, check_r, record

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


def test_growth_32_appends_of_8_digit_cache(cq, orc):
    m, p, count = 262147, 8, 32
    b = cq.Basis(m, p * count)
    b.enable_digit_cache()
    Qo = np.zeros((m, 0), order="F")
    Ro = np.zeros((0, 0))
    G = np.zeros((0, 0))  # Gramian of the GPU basis so far
    worst = 0.0
    for k in range(count):
        blk, eta = synth.update_block(Qo if k else None, m, p, k, seed=3)
        st, info = b.append(cq.to_colmajor(blk))
        Qn, Bn, Rn, sto, info_o = orc.cholqr_update(Qo, blk, min_iter=2)
        assert st == sto and st >= 0, (k, st, info, info_o)
        q = Qo.shape[1]
        Qg = b.Q().cpu().numpy()
        Rg = b.R().cpu().numpy()
        assert Qg.shape == (m, q + p)
        Qnew = Qg[:, q:]
        # orthogonality of the whole basis
        C = Qg.T @ Qnew
        G2 = np.zeros((q + p, q + p))
        G2[:q, :q] = G
        G2[:, q:] = C
        G2[q:, :q] = C[:q].T
        G = G2
        orth = float(np.linalg.norm(G - np.eye(q + p)))
        record("orthogonality (||Q^T Q - I||_F / 1e-13)", orth, ORTH_GATE, f"growth m={m} append {k}")
        assert orth <= ORTH_GATE, (k, orth)
        worst = max(worst, orth)
        # residual of the new block
        res = np.linalg.norm(blk - Qg @ Rg[: q + p, q:q + p]) / np.linalg.norm(blk)
        assert res <= 1e-13, (k, res)
        # the oracle's factors, entry by entry
        Qo = np.asfortranarray(np.hstack([Qo, Qn]))
        Ro = np.block([[Ro, Bn], [np.zeros((p, q)), Rn]])
        sv = np.linalg.svd(Ro, compute_uv=False)
        kap = sv[0] / sv[-1]
        scale = max(np.max(np.abs(Rn)), np.max(np.abs(Bn)) if q else 0.0)
        dR = float(np.max(np.abs(Rg[: q + p, q:q + p] - Ro[:, q:])))
        dQ = float(np.max(np.abs(Qnew - Qn)))
        print(f"append {k}: q={q} eta={eta:.1e} iters={info['iters']}/{info_o.iters} "
              f"shifts={info['shifts']}/{info_o.shifts} orth={orth:.1e} dQ={dQ:.1e} dR={dR:.1e} "
              f"kappa={kap:.1e}")
        check_r(dR, kap, np.array([scale]), m, f"growth m={m} append {k}")
        check_q(dQ, kap, m, f"growth m={m} append {k}")
    assert b.cols == p * count
    print(f"largest ||Q^T Q - I||_F over the run: {worst:.2e}")
    b.close()
