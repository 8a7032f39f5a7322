"""Host logic of the row-sharded factorisation on CPU (gloo, world size 2).

Each rank holds a contiguous row shard of A.  The product's TorchDistReducer
gathers the ranks' blocks in rank order; summing the gathered Gramian
partials in rank order (what the library's kernel does) gives, on both
ranks, bitwise the Gramian a single process forms from the same shards in
the same order, and that sum is the full Gramian within the FP64 dot-product
bound.  A rank whose peer never joins the exchange gets a failure from its
reducer callback (the library then returns CQR_ERR_REDUCE) instead of
waiting forever.  The oracle forms the shards' Gramians (test
infrastructure); no GPU is used.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, mode, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import datetime
    import torch.distributed as dist
    from paper_2507_07788_gb300 import synth
    from paper_2507_07788_gb300.sharded import TorchDistReducer, split_rows
    import oracle
    timeout = datetime.timedelta(seconds=6 if mode == "peer_absent" else 60)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timeout)
    try:
        m, n = 5003, 12
        red = TorchDistReducer(capacity=n * n, device="cpu")
        if mode == "gram":
            A = synth.test_matrix(m, n, 1e6, rep=3)
            r0, r1 = split_rows(m, world)[rank]
            X = oracle.gram(np.asfortranarray(A[r0:r1]))
            red.send[: n * n] = torch.from_numpy(X.reshape(-1, order="F").copy())
            rc = red._cb(None, n * n, None)
            blocks = red.recv[: world * n * n].numpy().reshape(world, n * n)
            s = blocks[0].copy()
            for r in range(1, world):
                s = s + blocks[r]
            out.put((rank, rc, s.tobytes(), [b.tobytes() for b in blocks]))
        else:  # rank 1 never joins the exchange
            if rank == 0:
                rc = red._cb(None, n * n, None)
                out.put((rank, rc, type(red.error).__name__, None))
            else:
                out.put((rank, None, None, None))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(world, mode):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, mode, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r = q.get(timeout=120)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    return res


def test_split_rows():
    from paper_2507_07788_gb300.sharded import split_rows
    assert split_rows(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert split_rows(7, 1) == [(0, 7)]
    with pytest.raises(ValueError):
        split_rows(2, 3)


def test_rank_ordered_gramian_matches_one_process(orc):
    from paper_2507_07788_gb300 import synth
    from paper_2507_07788_gb300.sharded import split_rows
    world = 2
    res = _run(world, "gram")
    m, n = 5003, 12
    A = synth.test_matrix(m, n, 1e6, rep=3)
    shards = [orc.gram(np.asfortranarray(A[r0:r1])) for r0, r1 in split_rows(m, world)]
    one = shards[0].reshape(-1, order="F").copy()
    for X in shards[1:]:
        one = one + X.reshape(-1, order="F")
    for r in range(world):
        rank, rc, s, blocks = res[r]
        assert rc == 0
        # the gathered blocks are the ranks' own partials, in rank order
        for k in range(world):
            assert blocks[k] == shards[k].reshape(-1, order="F").tobytes()
        # bitwise the one-process rank-ordered sum, on every rank
        assert s == one.tobytes()
    # and the full Gramian within the FP64 dot-product bound
    Xg = np.frombuffer(res[0][2]).reshape(n, n, order="F")
    absA = np.abs(A)
    u = 2.0 ** -53
    assert np.all(np.abs(Xg - orc.gram(A)) <= 2 * m * u * (absA.T @ absA))


def test_absent_peer_fails_the_exchange():
    res = _run(2, "peer_absent")
    rank, rc, err, _ = res[0]
    assert rc == 1 and err is not None
