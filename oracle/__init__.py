"""Plain FP64 CPU oracle for shifted Cholesky QR — TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  The product path (the CUDA library and
its Python binding) never imports it, and the two share no code.

The arithmetic lives in ``cholqr_oracle.c`` (plain C, IEEE double, sums in
index order, compiled with ``-ffp-contract=off``).  This module only builds it
with gcc and marshals numpy arrays (column-major, float64) through ctypes.

Function to paper map (arXiv 2507.07788):
  gram, chol, trsm, trmm ..... the steps of Alg. 1 (Sec. 2.1)
  shift ...................... Alg. 1 (sigma formula, 2u floor)
  update_shift ............... Alg. 2 (first shift of the update)
  cholqr ..................... Alg. 1 (+ the sCholQR3 first-pass shift, Sec. 4.1)
  cholqr_update .............. Alg. 2 (Sec. 2.2), Proposition 2.1
  pncholqr ................... Alg. 3 (Sec. 2.3)
  loo, rrr, rcr .............. the metrics of Sec. 4.1
  householder_qr ............. textbook checker (unique R with positive diagonal)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cholqr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, NOT_CONVERGED, ERR_BREAKDOWN = 0, 1, -2
SHIFT_SCHOLQR3, SHIFT_ON_BREAKDOWN, SHIFT_NONE, SHIFT_SCHOLQR3_STRICT, SHIFT_ISCHOLQR = 0, 1, 2, 3, 4
STOP_FROB_TOL, STOP_U_SQRT_N = 0, 1
U = 2.0 ** -53


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/liboracle.so (idempotent)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                              os.path.getmtime(os.path.join(_HERE, "cholqr_oracle.h")))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-o", tmp, _SRC, "-lm"], cwd=_HERE)
    os.replace(tmp, _LIB)
    return _LIB


class _Opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("min_iter", C.c_int),
                ("shift_policy", C.c_int), ("stop_rule", C.c_int), ("max_escalations", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("chol_attempts", C.c_int), ("shifts", C.c_int),
                ("escalations", C.c_int), ("sigma_first", C.c_double), ("sigma_last", C.c_double),
                ("orth_frob", C.c_double), ("proj_frob", C.c_double)]


@dataclass
class Info:
    iters: int
    chol_attempts: int
    shifts: int
    escalations: int
    sigma_first: float
    sigma_last: float
    orth_frob: float
    proj_frob: float

    @staticmethod
    def of(c: _Info) -> "Info":
        return Info(c.iters, c.chol_attempts, c.shifts, c.escalations, c.sigma_first,
                    c.sigma_last, c.orth_frob, c.proj_frob)


_lib = None
_P = C.POINTER(C.c_double)
_I64 = C.c_int64


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        d = C.c_double
        sig = {
            "orc_default_opts": (None, [C.POINTER(_Opts)]),
            "orc_gram": (None, [_I64, _I64, _P, _I64, _P, _I64]),
            "orc_gemm_tn": (None, [_I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64]),
            "orc_chol": (C.c_int, [_I64, _P, _I64, d, _P, _I64]),
            "orc_trsm_runn": (None, [_I64, _I64, _P, _I64, _P, _I64, _P, _I64]),
            "orc_trmm_upper": (None, [_I64, _P, _I64, _P, _I64, _P, _I64]),
            "orc_frob_minus_identity": (d, [_I64, _P, _I64]),
            "orc_sym_eigvals": (C.c_int, [_I64, _P, _I64, _P]),
            "orc_sym_norm2": (d, [_I64, _P, _I64]),
            "orc_shift": (d, [_I64, _I64, d]),
            "orc_update_shift": (d, [_I64, _I64, _I64, d]),
            "orc_cholqr": (C.c_int, [C.POINTER(_Opts), _I64, _I64, _P, _I64, _P, _I64, _P, _I64,
                                     C.POINTER(_Info)]),
            "orc_cholqr_update": (C.c_int, [C.POINTER(_Opts), _I64, _I64, _P, _I64, _I64, _P, _I64,
                                            _P, _I64, _P, _I64, _P, _I64, C.POINTER(_Info)]),
            "orc_pncholqr": (C.c_int, [C.POINTER(_Opts), _I64, _I64, _I64, _P, _I64, _P, _I64, _P,
                                       _I64, C.POINTER(_Info)]),
            "orc_householder_qr": (None, [_I64, _I64, _P, _I64, _P, _I64, _P, _I64]),
            "orc_loo": (d, [_I64, _I64, _P, _I64]),
            "orc_loo_frob": (d, [_I64, _I64, _P, _I64]),
            "orc_rrr": (d, [_I64, _I64, _P, _I64, _P, _I64, _P, _I64]),
            "orc_rcr": (d, [_I64, _I64, _P, _I64, _P, _I64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _f(a) -> np.ndarray:
    """Column-major float64 copy-or-view."""
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(_P)


def _ld(a: np.ndarray) -> int:
    return max(1, a.shape[0])


def opts(tol=1e-13, max_iter=10, min_iter=0, shift_policy=SHIFT_SCHOLQR3,
         stop_rule=STOP_FROB_TOL, max_escalations=40) -> _Opts:
    return _Opts(tol, max_iter, min_iter, shift_policy, stop_rule, max_escalations)


def gram(A) -> np.ndarray:
    A = _f(A)
    m, n = A.shape
    X = np.zeros((n, n), order="F")
    _load().orc_gram(m, n, _p(A), _ld(A), _p(X), max(1, n))
    return X


def gemm_tn(A, B) -> np.ndarray:
    A, B = _f(A), _f(B)
    m, p = A.shape
    q = B.shape[1]
    Cm = np.zeros((p, q), order="F")
    _load().orc_gemm_tn(m, p, q, _p(A), _ld(A), _p(B), _ld(B), _p(Cm), max(1, p))
    return Cm


def chol(X, sigma: float = 0.0):
    """Returns (R, rc): rc = 0 on success, else 1-based index of the failed pivot."""
    X = _f(X)
    n = X.shape[0]
    R = np.zeros((n, n), order="F")
    rc = _load().orc_chol(n, _p(X), max(1, n), float(sigma), _p(R), max(1, n))
    return R, rc


def trsm(A, R) -> np.ndarray:
    A, R = _f(A), _f(R)
    m, n = A.shape
    Q = np.zeros((m, n), order="F")
    _load().orc_trsm_runn(m, n, _p(A), _ld(A), _p(R), max(1, n), _p(Q), _ld(Q))
    return Q


def trmm_upper(T, R) -> np.ndarray:
    T, R = _f(T), _f(R)
    n = T.shape[0]
    Cm = np.zeros((n, n), order="F")
    _load().orc_trmm_upper(n, _p(T), max(1, n), _p(R), max(1, n), _p(Cm), max(1, n))
    return Cm


def frob_minus_identity(X) -> float:
    X = _f(X)
    return _load().orc_frob_minus_identity(X.shape[0], _p(X), max(1, X.shape[0]))


def sym_eigvals(X) -> np.ndarray:
    X = _f(X)
    n = X.shape[0]
    w = np.zeros(n)
    _load().orc_sym_eigvals(n, _p(X), max(1, n), _p(w))
    return np.sort(w)


def sym_norm2(X) -> float:
    X = _f(X)
    return _load().orc_sym_norm2(X.shape[0], _p(X), max(1, X.shape[0]))


def shift(m: int, n: int, normX: float) -> float:
    return _load().orc_shift(m, n, float(normX))


def update_shift(m: int, q: int, p: int, normX: float) -> float:
    return _load().orc_update_shift(m, q, p, float(normX))


def cholqr(A, o: _Opts | None = None, **kw):
    """Alg. 1 family.  Returns (Q, R, status, Info)."""
    A = _f(A)
    m, n = A.shape
    o = o or opts(**kw)
    Q = np.zeros((m, n), order="F")
    R = np.zeros((n, n), order="F")
    inf = _Info()
    st = _load().orc_cholqr(C.byref(o), m, n, _p(A), _ld(A), _p(Q), _ld(Q), _p(R), max(1, n),
                            C.byref(inf))
    return Q, R, st, Info.of(inf)


def cholqr_update(Qin, A_in, o: _Opts | None = None, **kw):
    """Alg. 2.  Returns (Q, B, R, status, Info) with [Qin Q][[Rin,B],[0,R]] = [Ain_prev A_in]."""
    A_in = _f(A_in)
    m, p = A_in.shape
    Qin = _f(Qin) if Qin is not None else np.zeros((m, 0), order="F")
    q = Qin.shape[1]
    o = o or opts(**kw)
    Q = np.zeros((m, p), order="F")
    B = np.zeros((max(q, 1), p), order="F")
    R = np.zeros((p, p), order="F")
    inf = _Info()
    qin_ptr = _p(Qin) if q > 0 else _p(np.zeros((1, 1), order="F"))
    st = _load().orc_cholqr_update(C.byref(o), m, q, qin_ptr, max(1, m), p, _p(A_in), _ld(A_in),
                                   _p(Q), _ld(Q), _p(B), max(1, q), _p(R), max(1, p), C.byref(inf))
    return Q, B[:q, :], R, st, Info.of(inf)


def pncholqr(A, r: int, o: _Opts | None = None, **kw):
    """Alg. 3 with r panels.  Returns (Q, R, status, Info)."""
    A = _f(A)
    m, n = A.shape
    o = o or opts(**kw)
    Q = np.zeros((m, n), order="F")
    R = np.zeros((n, n), order="F")
    inf = _Info()
    st = _load().orc_pncholqr(C.byref(o), m, n, int(r), _p(A), _ld(A), _p(Q), _ld(Q), _p(R),
                              max(1, n), C.byref(inf))
    return Q, R, st, Info.of(inf)


def householder_qr(A):
    A = _f(A)
    m, n = A.shape
    Q = np.zeros((m, n), order="F")
    R = np.zeros((n, n), order="F")
    _load().orc_householder_qr(m, n, _p(A), _ld(A), _p(Q), _ld(Q), _p(R), max(1, n))
    return Q, R


def loo(Q) -> float:
    Q = _f(Q)
    return _load().orc_loo(Q.shape[0], Q.shape[1], _p(Q), _ld(Q))


def loo_frob(Q) -> float:
    Q = _f(Q)
    return _load().orc_loo_frob(Q.shape[0], Q.shape[1], _p(Q), _ld(Q))


def rrr(A, Q, R) -> float:
    A, Q, R = _f(A), _f(Q), _f(R)
    m, n = A.shape
    return _load().orc_rrr(m, n, _p(A), _ld(A), _p(Q), _ld(Q), _p(R), max(1, n))


def rcr(A, R) -> float:
    A, R = _f(A), _f(R)
    m, n = A.shape
    return _load().orc_rcr(m, n, _p(A), _ld(A), _p(R), max(1, n))
