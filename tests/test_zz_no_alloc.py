"""cholqr_factor_noalloc, the entry point for callers that cannot allocate
device memory (all scratch in the library's fixed 8 MiB device array, n <= 64).

It is called through the C ABI and its Q and R are checked against those of
cholqr_factor on the same input, with the parity tolerances of
test_gpu_factor.py, for two calls in a row on different inputs: the second
call starts from the array contents the first call left behind.  This file
is collected last so that a failure here comes after every other test.
"""
import ctypes as C
import math

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


def q_tol(kappa, m, n):
    return max(1e-12, 20.0 * kappa * U * math.sqrt(n) / math.sqrt(m))


def r_tol(kappa, n, R):
    return 20.0 * max(kappa, 1.0) * U * math.sqrt(n) * np.max(np.abs(R))


def call(cq, fn, A):
    m, n = A.shape
    dA = cq.to_colmajor(A)
    dQ = cq.colmajor(m, n)
    dR = cq.colmajor(n, n)
    info = cq.Info()
    st = fn(None, m, n, dA.data_ptr(), m, dQ.data_ptr(), m, dR.data_ptr(), n, C.byref(info),
            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return dQ.cpu().numpy(), dR.cpu().numpy(), st, info.as_dict()


def test_noalloc_matches_factor_two_calls_in_a_row(cq):
    cases = [(40013, 64, 1e12, 0), (20037, 20, 1e8, 1)]
    for m, n, kappa, rep in cases:
        A = synth.test_matrix(m, n, kappa, rep=rep)
        Qn, Rn, stn, infon = call(cq, cq.cholqr_factor_noalloc, A)
        Qf, Rf, stf, infof = call(cq, cq.cholqr_factor, A)
        assert stn == stf == cq.OK, (stn, stf)
        assert infon["iters"] == infof["iters"]
        assert np.max(np.abs(Rn - Rf)) <= r_tol(kappa, n, Rf)
        assert np.max(np.abs(Qn - Qf)) <= q_tol(kappa, m, n)


def test_noalloc_rejects_n_beyond_limit(cq):
    info = cq.Info()
    st = cq.cholqr_factor_noalloc(None, 1000, 65, C.c_void_p(0x100000), 1000, C.c_void_p(0x900000),
                                  1000, C.c_void_p(0x2000000), 65, C.byref(info), None)
    assert st == cq.ERR_CAPACITY
