"""The Gramian X = A^T A (Alg. 1) as the library forms it
(cholqr_gram): tensor-core digit arithmetic (Ozaki splitting) for n <= 128
(emulation AUTO: the tcgen05 kernel for 33 <= n <= 64 and the warp-level
mma.sync kernels elsewhere; emulation TCGEN05: the tcgen05 kernel for
17 <= n <= 64; the tcgen05 kernel needs a 16-byte aligned block with an
even leading dimension, the mma.sync kernel forms the others) and
FP64 CUDA cores with emulation OFF, against the oracle's FP64 triple loop.
The tcgen05 and mma.sync kernels form the same exact digit products, but
each CTA splits X between its partial P and P^T differently (the tcgen05
kernel forms some off-diagonal digit blocks transposed), and each partial
entry is rounded once before the FP64 reduction.  Their results therefore
differ by the rounding of the G partials only: |X_1 - X_2| <= 4 (1 + G) u
(|A|^T |A|), far inside the dot-product bound for m >> G.

Tolerance: both sides are within the FP64 dot-product bound, so
|X_gpu - X_oracle|_ij <= 2 * gamma_m * (|A|^T |A|)_ij with gamma_m = m u / (1 - m u).
(The digit scheme's own error is below 2^-53 (|A|^T|A|)_ij plus 2^-56 of
the column maxima, far inside the bound.)"""
import itertools

import numpy as np
import pytest

from paper_2507_07788_gb300 import synth

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


def check(cq, orc, A, emu):
    m = A.shape[0]
    X = cq.gram(cq.to_colmajor(A), opts=cq.default_opts(emulation=emu)).cpu().numpy()
    Xo = orc.gram(A)
    absA = np.abs(A)
    bound = 2.0 * (m * U / (1 - m * U)) * (absA.T @ absA) + 1e-300
    assert np.all(np.abs(X - Xo) <= bound), np.max(np.abs(X - Xo) / bound)
    assert np.array_equal(X, X.T)
    return X


@pytest.mark.parametrize("emu", [0, 1, 2])
@pytest.mark.parametrize("m,n", [(1, 1), (17, 3), (128, 16), (129, 16), (5000, 20), (40000, 33),
                                 (60000, 64), (3000, 100), (5000, 65), (70000, 128)])
def test_gram_parity(cq, orc, emu, m, n):
    A = synth.test_matrix(m, n, 1e6, rep=2)
    check(cq, orc, A, emu)


def test_gram_exponent_growth_across_tiles(cq, orc):
    # every CTA sees several tiles whose column maxima grow from tile to tile
    m, n = 80000, 24
    rng = np.random.default_rng(3)
    scale = 10.0 ** (np.arange(m) // 128 % 7 - 3.0)[:, None] * 10.0 ** rng.uniform(-2, 2, size=(1, n))
    A = rng.standard_normal((m, n)) * scale
    check(cq, orc, A, 0)


def test_gram_extreme_column_scales(cq, orc):
    # column scales from 1e-150 to 1e150 (all squares representable)
    A = synth.test_matrix(20000, 8, 1e3, rep=13) * np.array([1.0, 1e-150, 1e150, 1e-30, 1e30, 3.0,
                                                             2.0 ** -400, 2.0 ** 450])
    check(cq, orc, A, 0)


def test_gram_exact_on_small_integers(cq):
    # small integer entries: every product and sum is exact in both paths
    rng = np.random.default_rng(4)
    A = rng.integers(-50, 51, size=(30000, 40)).astype(np.float64)
    Xe = cq.gram(cq.to_colmajor(A)).cpu().numpy()
    Xn = cq.gram(cq.to_colmajor(A), opts=cq.default_opts(emulation=cq.EMU_OFF)).cpu().numpy()
    ref = A.T @ A  # exact: |sum| < 2^53
    assert np.array_equal(Xe, ref) and np.array_equal(Xn, ref)


def test_gram_nan_propagates(cq):
    A = synth.gaussian(5000, 10, seed=1)
    A[77, 4] = np.nan
    X = cq.gram(cq.to_colmajor(A)).cpu().numpy()
    assert np.isnan(X).any()


def _rne(S: int, scale: int) -> float:
    """S * 2^scale rounded to FP64, ties to even (Python's int -> float
    conversion rounds to nearest even; the power-of-two scale is exact)."""
    return float(S) * 2.0 ** scale


@pytest.mark.parametrize("emu", [0, 2])
@pytest.mark.parametrize("n", [16, 40])
def test_gram_diagonal_is_correctly_rounded(cq, n, emu):
    # One 64-row tile: a single digit-Gramian CTA rounds each entry once from
    # the exact sum, and the reduction doubles P_jj exactly, so X_jj must be
    # the correctly rounded sum of squares.  Entries are M 2^(k_j - 25) with
    # |M| < 2^26: the squares are exact, their sum needs up to 58 bits, and
    # every element lies within the top 28 bits of its column (4 digits), so
    # no digit product is dropped.  The last entry of some columns is chosen
    # so that the exact sum is a tie between two doubles.
    rng = np.random.default_rng(11)
    m = 64
    M = rng.integers(-(2 ** 26) + 1, 2 ** 26, size=(m, n), dtype=np.int64)
    k = rng.integers(-40, 41, size=n)
    ties = 0
    for j in range(0, n, 2):
        # the last four entries (0..15 each; every residue is a sum of four
        # squares) are chosen so that the exact sum sits halfway between
        # two doubles
        S60 = sum(int(x) * int(x) for x in M[:-4, j])
        for e in itertools.product(range(16), repeat=4):
            S = S60 + sum(v * v for v in e)
            drop = S.bit_length() - 53
            if drop > 1 and S % (1 << drop) == 1 << (drop - 1):
                M[-4:, j] = e
                ties += 1
                break
    assert ties >= n // 2 - 2
    A = M.astype(np.float64) * np.exp2(k - 25)[None, :]
    X = cq.gram(cq.to_colmajor(A), opts=cq.default_opts(emulation=emu)).cpu().numpy()
    for j in range(n):
        S = sum(int(x) * int(x) for x in M[:, j])
        assert X[j, j] == _rne(S, 2 * (int(k[j]) - 25)), (j, X[j, j], _rne(S, 2 * (int(k[j]) - 25)))


@pytest.mark.parametrize("m,n,grow", [(1, 17, False), (63, 20, False), (4097, 33, False), (200003, 48, False),
                                      (1000000, 64, False), (300000, 64, True), (100000, 40, True)])
def test_tcgen05_and_mma_sync_gramians_agree(cq, orc, m, n, grow):
    # one tile, a ragged tile, several CTAs with ragged tails, the benchmark
    # size; with grow, column maxima that grow from tile to tile inside each
    # CTA (the rescaled integer sums)
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n))
    if grow:
        A *= 10.0 ** ((np.arange(m) // 64) % 9 - 4.0)[:, None] * 10.0 ** rng.uniform(-3, 3, size=(1, n))
    dA = cq.to_colmajor(A)
    Xt = cq.gram(dA, opts=cq.default_opts(emulation=cq.EMU_TCGEN05)).cpu().numpy()
    # the same block 8 bytes past a 16-byte boundary: the mma.sync kernel
    big = cq.colmajor(m + 1, n)
    big[1:].copy_(dA)
    Xl = cq.gram(big[1:]).cpu().numpy()
    assert np.array_equal(Xt, Xt.T)
    absA = np.abs(A)
    AtA = absA.T @ absA
    G = 2 * 152  # at most this many partials on either kernel
    assert np.all(np.abs(Xt - Xl) <= 4.0 * (1 + G) * U * AtA + 1e-300)
    if m <= 300000:
        Xo = orc.gram(A)
        bound = 2.0 * (m * U / (1 - m * U)) * AtA + 1e-300
        assert np.all(np.abs(Xt - Xo) <= bound)


def test_tcgen05_gramian_falls_back_on_unaligned_blocks(cq, orc):
    # an odd leading dimension and a block that starts 8 bytes past a 16-byte
    # boundary cannot be described to TMA: the mma.sync kernel forms them
    # (over the tcgen05 kernel's row groups, so the partials differ from the
    # default run's and the results agree within their rounding)
    m, n, ld = 20001, 40, 20003
    A = synth.test_matrix(m + 1, n, 1e4, rep=6)
    big = cq.colmajor(ld, n)
    big.zero_()
    big[: m + 1].copy_(torch.from_numpy(A))
    for view, ref in ((big[:m], A[:m]), (big[1: m + 1], A[1:])):
        X = cq.gram(view, opts=cq.default_opts(emulation=cq.EMU_TCGEN05)).cpu().numpy()
        Xl = cq.gram(view).cpu().numpy()
        absA = np.abs(ref)
        AtA = absA.T @ absA
        assert np.all(np.abs(X - Xl) <= 4.0 * (1 + 2 * 152) * U * AtA + 1e-300)
        Xo = orc.gram(np.asfortranarray(ref))
        assert np.all(np.abs(X - Xo) <= 2.0 * (m * U / (1 - m * U)) * AtA + 1e-300)
