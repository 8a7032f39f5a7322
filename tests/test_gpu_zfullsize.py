"""Parity at the benchmark's full size and launch configuration: sCholQR3 of
the 1e6 x 64 matrix with kappa = 1e12 (A = U diag(s) V^T, the benchmark's
own seed) under the default options, which run the chunked tensor-core pass
pipeline.  Q and R are compared with the oracle's sCholQR3 of the same matrix
entry by entry (about 15 s of oracle time) within the bounds of
tests/parity.py; the oracle's Gramian of A is compared with the library's
entry by entry, and the first shift with the one sized from it; the
orthogonality, residual and shape of R are checked outright.  The
mixed-precision variant (reduced-digit first Gramian) is compared with the
same oracle factors."""
import numpy as np
import pytest

from paper_2507_07788_gb300 import synth
from parity import check_orth, check_q, check_r

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module")
def cq():
    import paper_2507_07788_gb300 as cq
    from paper_2507_07788_gb300 import _build
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return cq


def test_benchmark_size_factorisation(cq, orc):
    m, n, kappa = 1_000_000, 64, 1e12
    A = synth.test_matrix(m, n, kappa, rep=0)
    dA = cq.to_colmajor(A)
    res = cq.factor(dA)
    torch.cuda.synchronize()
    Q, R = res.Q.cpu().numpy(), res.R.cpu().numpy()
    # the unshifted second pass sits at the breakdown threshold on this
    # matrix: 3 passes, or 4 after a recomputed shift
    assert res.status == cq.OK and res.info["iters"] in (3, 4), res.info
    check_orth(Q, "benchmark size")
    assert orc.rrr(A, Q, R) <= 1e-13
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)

    # the oracle's sCholQR3 of the same matrix, entry by entry (its
    # sequentially summed Gramians may take more passes to pass the stop
    # test, reading 16 of the design; the factors are unique all the same)
    Qo, Ro, sto, info_o = orc.cholqr(A)
    assert sto == cq.OK
    check_q(float(np.max(np.abs(Q - Qo))), kappa, m, "benchmark size 1e6x64")
    check_r(float(np.max(np.abs(R - Ro))), kappa, Ro, m, "benchmark size 1e6x64")

    # the mixed-precision variant on the same matrix against the same oracle
    # factors, with its first shift from the reduced-digit Gramian's bound
    mx = cq.factor(dA, opts=cq.default_opts(precision=cq.PREC_MIXED), check=False)
    torch.cuda.synchronize()
    assert mx.status == cq.OK, mx.info
    Qm, Rm = mx.Q.cpu().numpy(), mx.R.cpu().numpy()
    check_orth(Qm, "mixed benchmark size")
    assert orc.rrr(A, Qm, Rm) <= 1e-13
    check_q(float(np.max(np.abs(Qm - Qo))), kappa, m, "mixed benchmark size 1e6x64")
    check_r(float(np.max(np.abs(Rm - Ro))), kappa, Ro, m, "mixed benchmark size 1e6x64")
    assert mx.info["iters"] <= res.info["iters"], (mx.info, res.info)
    del Qo, Qm

    # the oracle's Gramian of A against the library's, every entry within
    # the FP64 dot-product bound, and the first shift from its norm
    Xo = orc.gram(A)
    Xg = cq.gram(dA).cpu().numpy()
    absA = np.abs(A)
    bound = 2.0 * (m * U / (1 - m * U)) * (absA.T @ absA)
    assert np.all(np.abs(Xg - Xo) <= bound), float(np.max(np.abs(Xg - Xo) / bound))
    assert np.array_equal(Xg, Xg.T)
    assert res.info["sigma_first"] == pytest.approx(orc.shift(m, n, orc.sym_norm2(Xo)), rel=1e-2)
