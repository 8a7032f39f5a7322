"""cholqr_factor_noalloc, the entry point for callers that cannot allocate
device memory: processes whose device memory already belongs to their own
allocator or budget, and loops that must not risk an allocation inside a
call.  All of its scratch is the library's fixed 8 MiB device array (n <= 64).

It runs the FP64 CUDA-core path of cholqr_factor (the path cholqr_factor
takes with emulation = CQR_EMU_OFF), so its Q and R must equal that call's
bit for bit; they are also checked against cholqr_factor's default path and
against the oracle, with the parity tolerances of tests/parity.py, for calls
in a row on different inputs (each call starts from the array contents the
previous one left behind), in place, with a non-default shift policy, and
through the max_iter exit.  This file is collected last so that a failure
here comes after every other test; it passes alone in a fresh process too.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2507_07788_gb300 import synth
from parity import check_q, check_r

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


def call(cq, fn, A, opts=None, inplace=False):
    m, n = A.shape
    dA = cq.to_colmajor(A)
    dQ = dA if inplace else cq.colmajor(m, n)
    dR = cq.colmajor(n, n)
    info = cq.Info()
    st = fn(C.byref(opts) if opts is not None else None, m, n, dA.data_ptr(), m, dQ.data_ptr(), m,
            dR.data_ptr(), n, C.byref(info), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return dQ.cpu().numpy(), dR.cpu().numpy(), st, info.as_dict()


def test_noalloc_two_calls_in_a_row(cq, orc):
    cases = [(40013, 64, 1e12, 0), (20037, 20, 1e8, 1)]
    off = cq.default_opts(emulation=cq.EMU_OFF)
    for m, n, kappa, rep in cases:
        A = synth.test_matrix(m, n, kappa, rep=rep)
        Qn, Rn, stn, infon = call(cq, cq.cholqr_factor_noalloc, A)
        Qe, Re, ste, infoe = call(cq, cq.cholqr_factor, A, opts=off)
        Qf, Rf, stf, infof = call(cq, cq.cholqr_factor, A)
        Qo, Ro, sto, info_o = orc.cholqr(A)
        assert stn == ste == stf == sto == cq.OK, (stn, ste, stf, sto)
        # the same kernels in the same order as the FP64 path of cholqr_factor
        assert np.array_equal(Qn, Qe) and np.array_equal(Rn, Re)
        assert infon == infoe
        # and within the parity bounds of the default path and of the oracle
        check_r(np.max(np.abs(Rn - Rf)), kappa, Rf, m, f"noalloc vs factor {m}x{n}")
        check_q(np.max(np.abs(Qn - Qf)), kappa, m, f"noalloc vs factor {m}x{n}")
        check_r(np.max(np.abs(Rn - Ro)), kappa, Ro, m, f"noalloc vs oracle {m}x{n}")
        check_q(np.max(np.abs(Qn - Qo)), kappa, m, f"noalloc vs oracle {m}x{n}")
        assert orc.loo_frob(Qn) <= 1e-13 and orc.rrr(A, Qn, Rn) <= 1e-13


def test_noalloc_in_place(cq, orc):
    m, n, kappa = 20011, 16, 1e10
    A = synth.test_matrix(m, n, kappa, rep=5)
    Qi, Ri, sti, infoi = call(cq, cq.cholqr_factor_noalloc, A, inplace=True)
    Qe, Re, ste, _ = call(cq, cq.cholqr_factor, A, opts=cq.default_opts(emulation=cq.EMU_OFF))
    Qo, Ro, sto, _ = orc.cholqr(A)
    assert sti == ste == sto == cq.OK
    assert np.array_equal(Qi, Qe) and np.array_equal(Ri, Re)
    check_q(np.max(np.abs(Qi - Qo)), kappa, m, "noalloc in place")
    check_r(np.max(np.abs(Ri - Ro)), kappa, Ro, m, "noalloc in place")


def test_noalloc_options_follow_the_fp64_path(cq):
    # isCholQR's reused shift on the paper's scale, and the max_iter exit of
    # the status poll: both equal to cholqr_factor's FP64 path bit for bit
    A = synth.test_matrix(20037, 20, 1e12, rep=2, paper_scale=True)
    for kw, want in ((dict(shift_policy=cq.SHIFT_ISCHOLQR), None),
                     (dict(max_iter=1), cq.NOT_CONVERGED),
                     (dict(max_iter=5, min_iter=4), cq.OK)):
        o = cq.default_opts(**kw)
        Qn, Rn, stn, infon = call(cq, cq.cholqr_factor_noalloc, A, opts=o)
        Qe, Re, ste, infoe = call(cq, cq.cholqr_factor, A, opts=cq.default_opts(emulation=cq.EMU_OFF, **kw))
        assert stn == ste, (kw, stn, ste)
        if want is not None:
            assert stn == want, (kw, stn)
        assert infon == infoe, kw
        assert np.array_equal(Qn, Qe) and np.array_equal(Rn, Re), kw


def test_noalloc_rejects_mixed_and_n_beyond_limit(cq):
    info = cq.Info()
    A = synth.test_matrix(3000, 8, 1e3)
    o = cq.default_opts(precision=cq.PREC_MIXED)
    _, _, st, _ = call(cq, cq.cholqr_factor_noalloc, A, opts=o)
    assert st == cq.ERR_INVALID
    st = cq.cholqr_factor_noalloc(None, 1000, 65, C.c_void_p(0x100000), 1000, C.c_void_p(0x900000),
                                  1000, C.c_void_p(0x2000000), 65, C.byref(info), None)
    assert st == cq.ERR_CAPACITY
    # host memory is not an operand of this entry point
    Ah = np.asfortranarray(A)
    Qh = np.empty_like(Ah)
    Rh = np.empty((8, 8), order="F")
    st = cq.cholqr_factor_noalloc(None, 3000, 8, Ah.ctypes.data, 3000, Qh.ctypes.data, 3000,
                                  Rh.ctypes.data, 8, C.byref(info), None)
    assert st == cq.ERR_INVALID
