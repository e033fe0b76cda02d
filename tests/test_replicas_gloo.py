"""The N > 1 path of bench.py runs independent replicas (one whole domain per GPU, no sharding).
Two gloo ranks on the CPU exercise its coordination: the torchrun environment, the barrier, the
max-over-ranks time and the whole-job throughput (all ranks' cell-updates / slowest rank's time)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(ws), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local, pg = bench.dist_setup(ws, backend="gloo")
    bench.barrier(pg)
    seconds = 1.0 + 0.5 * r            # rank 1 is the slow one
    value, t = bench.replica_value(pg, w, 1000.0, seconds, device="cpu")
    q.put((r, w, value, t))
    pg.destroy_process_group()


@pytest.mark.parametrize("ws", [2])
def test_replicas_take_the_slowest_rank(ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in range(ws)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, value, t in out:
        assert w == ws
        assert t == pytest.approx(1.5)
        assert value == pytest.approx(ws * 1000.0 / 1.5)


def test_single_process_is_its_own_job():
    sys.path.insert(0, ROOT)
    import bench
    value, t = bench.replica_value(None, 1, 500.0, 2.0)
    assert (value, t) == (250.0, 2.0)
