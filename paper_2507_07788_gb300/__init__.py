"""GB300-native shifted Cholesky QR (sCholQR3 with recomputed shift) and the
Cholesky-QR updating scheme of arXiv 2507.07788, as a thin Python binding
over the C ABI of ``libcholqr.so`` (declared in ``include/cholqr.h``).

Every step of the method runs in the library's CUDA kernels; this module
only marshals arguments.  It has no CPU fallback: if the library is missing
the first call raises.  PyTorch supplies device memory and streams.

Matrices are FP64 and column-major: a CUDA tensor of shape (m, n) with
``stride(0) == 1`` (see :func:`colmajor`).

Low-level functions carry the C names (``cholqr_factor``, ``basis_create``,
``basis_append``, ``basis_free``...) and take raw pointers; :func:`factor`
and :class:`Basis` wrap them for tensors::

    import paper_2507_07788_gb300 as cq
    A = cq.to_colmajor(a)               # numpy (m, n) float64 -> CUDA tensor
    res = cq.factor(A)                  # sCholQR3: res.Q, res.R, res.status
    b = cq.Basis(m, n_max)              # growing basis (Alg. 2)
    b.enable_digit_cache()              # optional: tensor-core narrow appends
    st, info = b.append(cq.to_colmajor(block))
    Q, R = b.Q(), b.R()                 # device views of the basis
    res = cq.pn(A, r=4)                 # pnCholQR (Alg. 3)
    res = cq.factor_host(a)             # host buffers in, host Q and R out
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcholqr.so")

# status codes (cqr_status)
OK, NOT_CONVERGED = 0, 1
ERR_INVALID, ERR_BREAKDOWN, ERR_OOM, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT = -1, -2, -3, -4, -5, -6
ERR_REDUCE = -7
SHIFT_SCHOLQR3, SHIFT_ON_BREAKDOWN, SHIFT_NONE, SHIFT_SCHOLQR3_STRICT, SHIFT_ISCHOLQR = 0, 1, 2, 3, 4
STOP_FROB_TOL, STOP_U_SQRT_N = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
EMU_AUTO, EMU_OFF, EMU_TCGEN05 = 0, 1, 2
MAX_N, MAX_BASIS = 512, 1024


class Opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("min_iter", C.c_int32),
                ("update_min_iter", C.c_int32), ("precision", C.c_int32),
                ("shift_policy", C.c_int32), ("stop_rule", C.c_int32),
                ("max_escalations", C.c_int32), ("emulation", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("chol_attempts", C.c_int32), ("shifts", C.c_int32),
                ("escalations", C.c_int32), ("sigma_first", C.c_double),
                ("sigma_last", C.c_double), ("orth_frob", C.c_double), ("proj_frob", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Timing(C.Structure):
    _fields_ = [("kernel_launches", C.c_int64), ("sweep_launches", C.c_int64),
                ("sweep_ms", C.c_double), ("sweep_flops", C.c_double), ("sweep_bytes", C.c_double),
                ("fused_launches", C.c_int64), ("fused_ms", C.c_double),
                ("fused_flops", C.c_double), ("fused_bytes", C.c_double),
                ("solve_launches", C.c_int64), ("solve_ms", C.c_double),
                ("solve_flops", C.c_double), ("solve_bytes", C.c_double),
                ("gram_launches", C.c_int64), ("gram_ms", C.c_double),
                ("gram_flops", C.c_double), ("gram_bytes", C.c_double),
                ("tsolve_launches", C.c_int64), ("tsolve_ms", C.c_double),
                ("tsolve_flops", C.c_double), ("tsolve_bytes", C.c_double),
                ("tsolve_tc_flops", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerOpts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("batch_max", C.c_int32), ("hbm_budget_bytes", C.c_int64),
                ("small_rows", C.c_int64)]


class RequestResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("kind", C.c_int32), ("batched", C.c_int32),
                ("batch_size", C.c_int32), ("t_submit", C.c_double), ("t_start", C.c_double),
                ("t_done", C.c_double), ("info", Info)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "info"}
        d["info"] = self.info.as_dict()
        return d


ALLGATHER_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int64, C.c_void_p)


class Reducer(C.Structure):
    """cqr_reducer: exchange buffers and callback of a row-sharded factorisation."""
    _fields_ = [("world", C.c_int32), ("rank", C.c_int32), ("send", C.c_void_p), ("recv", C.c_void_p),
                ("capacity", C.c_int64), ("allgather", ALLGATHER_FN), ("ctx", C.c_void_p)]


class CholQRError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: status {status} ({status_string(status)})")


_lib = None
_I64, _VP, _P = C.c_int64, C.c_void_p, C.c_void_p

# name -> (restype, argtypes); the exported C ABI
_SIGNATURES = {
    "cqr_default_opts": (None, [C.POINTER(Opts)]),
    "cqr_status_string": (C.c_char_p, [C.c_int]),
    "cholqr_factor": (C.c_int, [C.POINTER(Opts), _I64, _I64, _P, _I64, _P, _I64, _P, _I64,
                                C.POINTER(Info), _VP]),
    "cholqr_factor_host": (C.c_int, [C.POINTER(Opts), _I64, _I64, _P, _I64, _P, _I64, _P, _I64,
                                     C.POINTER(Info), _VP]),
    "cholqr_gram": (C.c_int, [C.POINTER(Opts), _I64, _I64, _P, _I64, _P, _I64, _VP]),
    "cholqr_factor_sharded": (C.c_int, [C.POINTER(Opts), _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64,
                                        C.POINTER(Reducer), C.POINTER(Info), _VP]),
    "cholqr_pn": (C.c_int, [C.POINTER(Opts), _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64,
                            C.POINTER(Info), _VP]),
    "cholqr_factor_noalloc": (C.c_int, [C.POINTER(Opts), _I64, _I64, _P, _I64, _P, _I64, _P,
                                        _I64, C.POINTER(Info), _VP]),
    "basis_create": (C.c_int, [_I64, _I64, C.POINTER(Opts), _VP, C.POINTER(_VP)]),
    "basis_append": (C.c_int, [_VP, _I64, _P, _I64, C.POINTER(Info), _VP]),
    "basis_free": (C.c_int, [_VP]),
    "basis_enable_digit_cache": (C.c_int, [_VP, _VP]),
    "basis_cols": (_I64, [_VP]),
    "basis_rows": (_I64, [_VP]),
    "basis_capacity": (_I64, [_VP]),
    "basis_q": (C.c_int, [_VP, C.POINTER(_VP), C.POINTER(_I64)]),
    "basis_r": (C.c_int, [_VP, C.POINTER(_VP), C.POINTER(_I64)]),
    "cqr_server_default_opts": (None, [C.POINTER(ServerOpts)]),
    "cqr_server_create": (C.c_int, [C.POINTER(ServerOpts), C.POINTER(_VP)]),
    "cqr_server_submit_factor": (C.c_int, [_VP, _VP, _I64, _P, _I64, C.POINTER(Opts),
                                           C.POINTER(C.c_uint64)]),
    "cqr_server_submit_append": (C.c_int, [_VP, _VP, _I64, _P, _I64, C.POINTER(C.c_uint64)]),
    "cqr_server_wait": (C.c_int, [_VP, C.c_uint64, C.POINTER(RequestResult)]),
    "cqr_server_drain": (C.c_int, [_VP]),
    "cqr_server_now": (C.c_double, [_VP]),
    "cqr_server_destroy": (C.c_int, [_VP]),
    "cqr_timing_enable": (C.c_int, [C.c_int]),
    "cqr_timing_read": (C.c_int, [C.POINTER(Timing)]),
    "cqr_timing_reset": (None, []),
}


def lib():
    """Load libcholqr.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGNATURES)


def status_string(status: int) -> str:
    return lib().cqr_status_string(int(status)).decode()


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().cqr_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


# ----------------------------------------------------------------- raw C ABI

def cholqr_factor(opts, m, n, A, lda, Q, ldq, R, ldr, info, stream) -> int:
    return lib().cholqr_factor(opts, m, n, A, lda, Q, ldq, R, ldr, info, stream)


def cholqr_factor_host(opts, m, n, A, lda, Q, ldq, R, ldr, info, stream) -> int:
    return lib().cholqr_factor_host(opts, m, n, A, lda, Q, ldq, R, ldr, info, stream)


def cholqr_factor_noalloc(opts, m, n, A, lda, Q, ldq, R, ldr, info, stream) -> int:
    """cholqr_factor with all scratch in the library's fixed device array (no
    allocation; n <= 64); for callers that cannot allocate device memory."""
    return lib().cholqr_factor_noalloc(opts, m, n, A, lda, Q, ldq, R, ldr, info, stream)


def cholqr_factor_sharded(opts, m_local, m_total, n, A, lda, Q, ldq, R, ldr, reducer, info, stream) -> int:
    """Row-sharded sCholQR3 on this rank's rows (reducer: a Reducer structure);
    see paper_2507_07788_gb300.sharded for reducers and a tensor wrapper."""
    return lib().cholqr_factor_sharded(opts, m_local, m_total, n, A, lda, Q, ldq, R, ldr, reducer, info,
                                       stream)


def basis_create(m, n_max, opts, stream):
    h = _VP()
    st = lib().basis_create(m, n_max, opts, stream, C.byref(h))
    return st, h


def basis_append(b, p, A_in, lda, info, stream) -> int:
    return lib().basis_append(b, p, A_in, lda, info, stream)


def basis_free(b) -> int:
    return lib().basis_free(b)


def cqr_timing_enable(enable: bool) -> int:
    return lib().cqr_timing_enable(1 if enable else 0)


def cqr_timing_read() -> dict:
    t = Timing()
    st = lib().cqr_timing_read(C.byref(t))
    if st != OK:
        raise CholQRError(st, "cqr_timing_read")
    return t.as_dict()


def cqr_timing_reset() -> None:
    lib().cqr_timing_reset()


# ----------------------------------------------------------------- tensor helpers

def _torch():
    import torch
    return torch


def colmajor(m: int, n: int, device="cuda", dtype=None):
    """Uninitialised column-major (m, n) float64 tensor (stride (1, m))."""
    torch = _torch()
    return torch.empty((n, m), dtype=dtype or torch.float64, device=device).t()


def to_colmajor(x, device="cuda"):
    """Copy of x (numpy array or tensor) as a column-major float64 CUDA tensor."""
    torch = _torch()
    t = x if isinstance(x, torch.Tensor) else torch.from_numpy(x)
    out = colmajor(t.shape[0], t.shape[1], device=device)
    out.copy_(t.to(torch.float64))
    return out


def _check_colmajor(t, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or t.dim() != 2:
        raise TypeError(f"{name} must be a 2-D float64 tensor")
    if t.shape[0] > 1 and t.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1)")
    return max(t.stride(1), t.shape[0], 1)


def _stream_ptr(stream):
    if stream is None:
        return _torch().cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


@dataclass
class Result:
    Q: object
    R: object
    status: int
    info: dict


def factor(A, Q=None, R=None, opts: Opts | None = None, stream=None, check=True) -> Result:
    """QR of a column-major CUDA tensor A (m x n) by cholqr_factor.

    Q may be A (in place).  Returns Result(Q, R, status, info)."""
    torch = _torch()
    lda = _check_colmajor(A, "A")
    m, n = A.shape
    if Q is None:
        Q = colmajor(m, n, device=A.device)
    if R is None:
        R = colmajor(n, n, device=A.device)
    ldq = _check_colmajor(Q, "Q")
    ldr = _check_colmajor(R, "R")
    info = Info()
    with torch.cuda.device(A.device):
        st = lib().cholqr_factor(C.byref(opts) if opts is not None else None, m, n, A.data_ptr(),
                                 lda, Q.data_ptr(), ldq, R.data_ptr(), ldr, C.byref(info),
                                 _stream_ptr(stream))
    if check and st < 0:
        raise CholQRError(st, "cholqr_factor")
    return Result(Q, R, st, info.as_dict())


def pn(A, r: int, Q=None, R=None, opts: Opts | None = None, stream=None, check=True) -> Result:
    """pnCholQR (Alg. 3) of a column-major CUDA tensor A (m x n) in r column
    panels through cholqr_pn.  Returns Result(Q, R, status, info)."""
    torch = _torch()
    lda = _check_colmajor(A, "A")
    m, n = A.shape
    if Q is None:
        Q = colmajor(m, n, device=A.device)
    if R is None:
        R = colmajor(n, n, device=A.device)
    ldq = _check_colmajor(Q, "Q")
    ldr = _check_colmajor(R, "R")
    info = Info()
    with torch.cuda.device(A.device):
        st = lib().cholqr_pn(C.byref(opts) if opts is not None else None, m, n, int(r), A.data_ptr(),
                             lda, Q.data_ptr(), ldq, R.data_ptr(), ldr, C.byref(info),
                             _stream_ptr(stream))
    if check and st < 0:
        raise CholQRError(st, "cholqr_pn")
    return Result(Q, R, st, info.as_dict())


def gram(A, opts: Opts | None = None, stream=None):
    """X = A^T A of a column-major CUDA tensor through cholqr_gram."""
    torch = _torch()
    lda = _check_colmajor(A, "A")
    m, n = A.shape
    X = colmajor(n, n, device=A.device)
    with torch.cuda.device(A.device):
        st = lib().cholqr_gram(C.byref(opts) if opts is not None else None, m, n, A.data_ptr(), lda,
                               X.data_ptr(), n, _stream_ptr(stream))
    if st != OK:
        raise CholQRError(st, "cholqr_gram")
    return X


def factor_host(A, Q=None, R=None, opts: Opts | None = None, stream=None, check=True) -> Result:
    """QR of a host matrix (numpy array or CPU tensor, float64) through
    cholqr_factor_host: copies in, factors on the GPU, copies Q and R out.
    Q (m x n) and R (n x n) may be given as column-major host tensors (pinned
    memory gives full copy bandwidth); otherwise pinned ones are allocated.
    Returns host (CPU tensor) Q and R."""
    torch = _torch()
    t = A if isinstance(A, torch.Tensor) else torch.from_numpy(A)
    if t.dtype != torch.float64 or t.dim() != 2 or t.device.type != "cpu":
        raise TypeError("A must be a 2-D float64 host array")
    m, n = t.shape
    if t.stride(0) != 1:
        t = t.t().contiguous().t()
    lda = max(t.stride(1), m)
    if Q is None:
        Q = torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()
    if R is None:
        R = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
    for M, name, rows, cols in ((Q, "Q", m, n), (R, "R", n, n)):
        if (M.dtype != torch.float64 or M.device.type != "cpu" or tuple(M.shape) != (rows, cols)
                or M.stride(0) != 1 or (cols > 1 and M.stride(1) < rows)):
            raise TypeError(f"{name} must be a column-major {rows} x {cols} float64 host tensor")
    info = Info()
    st = lib().cholqr_factor_host(C.byref(opts) if opts is not None else None, m, n, t.data_ptr(),
                                  lda, Q.data_ptr(), max(Q.stride(1), m), R.data_ptr(),
                                  max(R.stride(1), n), C.byref(info), _stream_ptr(stream))
    if check and st < 0:
        raise CholQRError(st, "cholqr_factor_host")
    return Result(Q, R, st, info.as_dict())


class Basis:
    """A growing orthonormal basis on the device (basis_create / append / free)."""

    def __init__(self, m: int, n_max: int, opts: Opts | None = None, stream=None):
        self._stream = stream
        st, h = basis_create(m, n_max, C.byref(opts) if opts is not None else None,
                             _stream_ptr(stream))
        if st != OK:
            raise CholQRError(st, "basis_create")
        self._h = h
        self.m, self.n_max = m, n_max

    def append(self, A_in, stream=None, check=True):
        lda = _check_colmajor(A_in, "A_in")
        info = Info()
        st = basis_append(self._h, A_in.shape[1], A_in.data_ptr(), lda, C.byref(info),
                          _stream_ptr(stream if stream is not None else self._stream))
        if check and st < 0:
            raise CholQRError(st, "basis_append")
        return st, info.as_dict()

    def enable_digit_cache(self, stream=None):
        """basis_enable_digit_cache: keep the digits of the basis columns on the
        device so narrow appends to a tall basis form their cross Gramian on
        the tensor cores."""
        st = lib().basis_enable_digit_cache(self._h, _stream_ptr(stream if stream is not None else self._stream))
        if st != OK:
            raise CholQRError(st, "basis_enable_digit_cache")

    @property
    def cols(self) -> int:
        return lib().basis_cols(self._h)

    def _view(self, getter, rows, cols):
        torch = _torch()
        ptr, ld = _VP(), _I64()
        st = getter(self._h, C.byref(ptr), C.byref(ld))
        if st != OK:
            raise CholQRError(st, "basis accessor")
        return _device_view(ptr.value, rows, cols, ld.value)

    def Q(self):
        """Device view (m x q) of the basis vectors (valid until the next append/free)."""
        return self._view(lib().basis_q, self.m, self.cols)

    def R(self):
        """Device view (q x q) of the upper triangular factor."""
        q = self.cols
        return self._view(lib().basis_r, q, q)

    def close(self):
        if getattr(self, "_h", None):
            basis_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _device_view(ptr: int, rows: int, cols: int, ld: int):
    """Column-major float64 tensor viewing device memory owned elsewhere."""
    torch = _torch()
    if rows == 0 or cols == 0:
        return torch.empty((rows, cols), dtype=torch.float64, device="cuda")
    nbytes = 8 * (ld * (cols - 1) + rows)

    class _Arr:
        __cuda_array_interface__ = {"shape": (nbytes // 8,), "typestr": "<f8",
                                    "data": (ptr, False), "version": 3, "strides": None}

    flat = torch.as_tensor(_Arr(), device="cuda")
    return flat.as_strided((rows, cols), (1, ld))


class Server:
    """Continuous-batching request server over device-resident bases
    (cqr_server_*).  Submissions return tickets; wait() returns the result
    with its timestamps on the server clock.  The server reads a request's
    input until the request completes, so the binding holds the input tensor
    (and its basis) until wait(), drain() or close()."""

    def __init__(self, slots=4, batch_max=16, hbm_budget_bytes=8 << 30, small_rows=262144):
        o = ServerOpts(slots, batch_max, hbm_budget_bytes, small_rows)
        h = _VP()
        st = lib().cqr_server_create(C.byref(o), C.byref(h))
        if st != OK:
            raise CholQRError(st, "cqr_server_create")
        self._h = h
        self._held = {}

    def now(self) -> float:
        return lib().cqr_server_now(self._h)

    def submit_factor(self, basis: "Basis", A, opts: Opts | None = None) -> int:
        lda = _check_colmajor(A, "A")
        t = C.c_uint64()
        st = lib().cqr_server_submit_factor(self._h, basis._h, A.shape[1], A.data_ptr(), lda,
                                            C.byref(opts) if opts is not None else None, C.byref(t))
        if st != OK:
            raise CholQRError(st, "cqr_server_submit_factor")
        self._held[t.value] = (A, basis)
        return t.value

    def submit_append(self, basis: "Basis", A_in) -> int:
        lda = _check_colmajor(A_in, "A_in")
        t = C.c_uint64()
        st = lib().cqr_server_submit_append(self._h, basis._h, A_in.shape[1], A_in.data_ptr(), lda,
                                            C.byref(t))
        if st != OK:
            raise CholQRError(st, "cqr_server_submit_append")
        self._held[t.value] = (A_in, basis)
        return t.value

    def wait(self, ticket: int) -> dict:
        r = RequestResult()
        st = lib().cqr_server_wait(self._h, ticket, C.byref(r))
        if st != OK:
            raise CholQRError(st, "cqr_server_wait")
        self._held.pop(ticket, None)
        return r.as_dict()

    def drain(self) -> None:
        lib().cqr_server_drain(self._h)
        self._held.clear()

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().cqr_server_destroy(self._h)
            self._h = None
        self._held = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
