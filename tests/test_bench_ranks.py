"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): the
replica throughput takes the slowest rank's time and sums the ranks' work,
and the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, ms_local, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms, value = bench.replica_throughput(ms_local, ws, 1000, 8, "cpu")
        out.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = {0: 3.0, 1: 5.0}
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times[r], q)) for r in (0, 1)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 5.0                          # max over ranks
        assert value == pytest.approx(2 * 1000 * 8 / 5e-3)  # both ranks' work


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.replica_throughput(4.0, 1, 1000, 8, "cpu")
    assert ms == 4.0 and value == pytest.approx(1000 * 8 / 4e-3)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
