"""The seeded input generators on CPU: the test matrices have the singular
values Sec. 4.1 prescribes (log-spaced, condition number kappa; 1 down to
1/kappa by default, 1 up to kappa on the paper's scale), the update blocks
follow their recipe, and every input is a pure function of its seed."""
import math

import numpy as np
import pytest

from paper_2507_07788_gb300 import synth


@pytest.mark.parametrize("kappa", [1.0, 1e4, 1e8])
def test_singular_values_and_condition(kappa):
    m, n = 500, 12
    A = synth.test_matrix(m, n, kappa, rep=1)
    s = np.linalg.svd(A, compute_uv=False)
    want = np.logspace(0.0, -math.log10(kappa), n)
    assert np.allclose(s, want, rtol=1e-12 * max(kappa, 1.0) ** 0.5, atol=0)
    P = synth.test_matrix(m, n, kappa, rep=1, paper_scale=True)
    sp = np.linalg.svd(P, compute_uv=False)
    assert np.allclose(sp, want * kappa, rtol=1e-12 * max(kappa, 1.0) ** 0.5, atol=0)
    assert sp[0] == pytest.approx(kappa, rel=1e-12) and sp[-1] == pytest.approx(1.0, rel=1e-8)


def test_large_kappa_keeps_the_top_of_the_spectrum():
    # beyond 1/u only the large singular values are resolved by an SVD
    A = synth.test_matrix(300, 10, 1e20, rep=0, salt=1)
    s = np.linalg.svd(A, compute_uv=False)
    want = np.logspace(0.0, -20.0, 10)
    assert np.allclose(s[:4], want[:4], rtol=1e-10, atol=0)
    assert s[-1] < 1e-14


def test_column_major_and_seeded():
    A = synth.test_matrix(200, 7, 1e6, rep=3, salt=2)
    assert A.flags.f_contiguous and A.dtype == np.float64
    assert np.array_equal(A, synth.test_matrix(200, 7, 1e6, rep=3, salt=2))
    assert not np.array_equal(A, synth.test_matrix(200, 7, 1e6, rep=4, salt=2))
    assert not np.array_equal(A, synth.test_matrix(200, 7, 1e6, rep=3, salt=3))
    G = synth.gaussian(100, 3, seed=5)
    assert G.flags.f_contiguous and np.array_equal(G, synth.gaussian(100, 3, seed=5))
    U = synth.orthonormal(100, 6, seed=1)
    assert np.linalg.norm(U.T @ U - np.eye(6)) < 1e-14


def test_update_blocks_follow_the_recipe():
    m, p = 400, 4
    b0, eta0 = synth.update_block(None, m, p, 0, seed=2)
    assert eta0 == 1.0 and b0.shape == (m, p)
    Q, _ = np.linalg.qr(synth.gaussian(m, 6, seed=9))
    b1, eta1 = synth.update_block(Q, m, p, 1, seed=2)
    assert 1e-12 <= eta1 <= 1.0
    # the block is Q G 0.1 + N eta: its part outside span(Q) has size ~eta
    out = b1 - Q @ (Q.T @ b1)
    assert np.linalg.norm(out) / math.sqrt(m * p) == pytest.approx(eta1, rel=0.2)
    # and its part inside span(Q) is 0.1 G + eta Q^T N, of size ~sqrt(0.01 + eta^2)
    assert np.linalg.norm(Q.T @ b1) / math.sqrt(6 * p) == pytest.approx(math.hypot(0.1, eta1), rel=0.5)
    blocks, etas = synth.basis_growth_blocks(m, p, 3, seed=2)
    assert len(blocks) == 3 and etas[0] == 1.0 and all(1e-12 <= e <= 1.0 for e in etas[1:])
