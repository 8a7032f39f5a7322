"""Row-sharded sCholQR3 (communication-avoiding Cholesky QR, Sec. 1 of the
paper): the m rows are split into contiguous blocks, one per rank; each rank
calls ``cholqr_factor_sharded`` on its block, the library exchanges the n x n
Gramian partials of every pass through a reducer and sums them in rank order
with its own kernel, so every rank takes the same decisions and holds the
same R; the solves are row-local.

This module only marshals arguments and moves the exchange buffers: every
step of the factorisation runs in the library's kernels.  Two reducers:

* ``TorchDistReducer`` -- one rank per process, over ``torch.distributed``
  (NCCL for CUDA buffers): ``all_gather_into_tensor`` queued on the library's
  stream.
* ``LocalReducerGroup`` -- several ranks as threads of one process (for
  example one thread per GPU): each exchange synchronises the rank's stream,
  stages its block in host memory, waits for the other ranks at a barrier
  with a timeout, and copies the rank-ordered blocks back.  A rank that does
  not arrive within the timeout makes every waiting rank's call return
  CQR_ERR_REDUCE.

A reducer's ``allgather(count, stream)`` raises on failure; the callback
turns that into a nonzero return, which the library reports as
``ERR_REDUCE``.
"""
from __future__ import annotations

import ctypes as C
import threading

from . import (ALLGATHER_FN, CholQRError, Info, Opts, Reducer, Result, _check_colmajor, _stream_ptr, colmajor,
               lib)


def split_rows(m: int, world: int) -> list[tuple[int, int]]:
    """Contiguous row blocks [r0, r1) of m rows over `world` ranks; the first
    m % world ranks get one row more."""
    if world < 1 or m < world:
        raise ValueError("need 1 <= world <= m")
    base, extra = divmod(m, world)
    out, r0 = [], 0
    for r in range(world):
        r1 = r0 + base + (1 if r < extra else 0)
        out.append((r0, r1))
        r0 = r1
    return out


class _ReducerBase:
    """Owns the exchange buffers and the C callback of one rank."""

    def __init__(self, world: int, rank: int, capacity: int, device):
        import torch
        if not (0 <= rank < world):
            raise ValueError("need 0 <= rank < world")
        self.world, self.rank, self.capacity = int(world), int(rank), int(capacity)
        self.send = torch.zeros(self.capacity, dtype=torch.float64, device=device)
        self.recv = torch.zeros(self.world * self.capacity, dtype=torch.float64, device=device)
        self.error: BaseException | None = None
        self.calls = 0

        def cb(ctx, count, stream):
            try:
                self.calls += 1
                self.allgather(int(count), stream)
                return 0
            except BaseException as exc:  # reported to the library as a failure
                self.error = exc
                return 1

        self._cb = ALLGATHER_FN(cb)  # kept alive as long as the reducer
        self.struct = Reducer(self.world, self.rank, self.send.data_ptr(), self.recv.data_ptr(),
                              self.capacity, self._cb, None)

    def allgather(self, count: int, stream) -> None:  # pragma: no cover - abstract
        raise NotImplementedError


class TorchDistReducer(_ReducerBase):
    """One rank per process over torch.distributed (initialised by the caller).
    The gather is queued on the library's stream (NCCL for CUDA buffers)."""

    def __init__(self, capacity: int, device="cuda", group=None):
        import torch.distributed as dist
        self.group = group
        super().__init__(dist.get_world_size(group), dist.get_rank(group), capacity, device)

    def allgather(self, count: int, stream) -> None:
        import torch
        import torch.distributed as dist
        if count > self.capacity:
            raise ValueError("count beyond the reducer's capacity")
        if self.send.is_cuda and stream:
            s = torch.cuda.ExternalStream(stream, device=self.send.device)
            with torch.cuda.stream(s):
                dist.all_gather_into_tensor(self.recv[: self.world * count], self.send[:count], group=self.group)
        else:
            dist.all_gather_into_tensor(self.recv[: self.world * count], self.send[:count], group=self.group)


class LocalReducerGroup:
    """`world` ranks as threads of one process: ``reducer(rank)`` is the
    reducer each rank's thread passes to ``factor_sharded``."""

    def __init__(self, world: int, capacity: int, devices=None, timeout_s: float = 30.0):
        import numpy as np
        self.world, self.capacity, self.timeout_s = int(world), int(capacity), float(timeout_s)
        self._barrier = threading.Barrier(self.world)
        self._stage = np.zeros((self.world, self.capacity))
        devs = devices if devices is not None else ["cuda"] * self.world
        self._reducers = [_LocalReducer(self, r, devs[r]) for r in range(self.world)]

    def reducer(self, rank: int) -> "_LocalReducer":
        return self._reducers[rank]

    def abort(self) -> None:
        """Breaks the barrier: every rank waiting in an exchange fails."""
        self._barrier.abort()


class _LocalReducer(_ReducerBase):
    def __init__(self, group: LocalReducerGroup, rank: int, device):
        self.group = group
        super().__init__(group.world, rank, group.capacity, device)

    def allgather(self, count: int, stream) -> None:
        import torch
        g = self.group
        if count > self.capacity:
            raise ValueError("count beyond the reducer's capacity")
        s = torch.cuda.ExternalStream(stream, device=self.send.device) if stream else \
            torch.cuda.current_stream(self.send.device)
        s.synchronize()  # the library's local block is in `send`
        g._stage[self.rank, :count] = self.send[:count].cpu().numpy()
        g._barrier.wait(timeout=g.timeout_s)  # every block staged
        blocks = torch.from_numpy(g._stage[:, :count].reshape(-1).copy())
        with torch.cuda.stream(s):
            self.recv[: self.world * count].copy_(blocks.to(self.recv.device, non_blocking=False))
        s.synchronize()
        g._barrier.wait(timeout=g.timeout_s)  # every rank has read the stage


def factor_sharded(A_local, m_total: int, reducer: _ReducerBase, Q=None, R=None, opts: Opts | None = None,
                   stream=None, check=True) -> Result:
    """sCholQR3 of this rank's row block A_local (column-major CUDA tensor,
    m_local x n) of a matrix with m_total rows.  Returns this rank's rows of Q
    and the full R.  With check, a failed exchange raises the reducer's own
    exception, any other error a CholQRError."""
    import torch
    lda = _check_colmajor(A_local, "A")
    m, n = A_local.shape
    if Q is None:
        Q = colmajor(m, n, device=A_local.device)
    if R is None:
        R = colmajor(n, n, device=A_local.device)
    ldq = _check_colmajor(Q, "Q")
    ldr = _check_colmajor(R, "R")
    info = Info()
    with torch.cuda.device(A_local.device):
        st = lib().cholqr_factor_sharded(C.byref(opts) if opts is not None else None, m, int(m_total), n,
                                         A_local.data_ptr(), lda, Q.data_ptr(), ldq, R.data_ptr(), ldr,
                                         C.byref(reducer.struct), C.byref(info), _stream_ptr(stream))
    if check and st < 0:
        if reducer.error is not None:
            raise reducer.error
        raise CholQRError(st, "cholqr_factor_sharded")
    return Result(Q, R, st, info.as_dict())
