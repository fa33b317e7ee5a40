"""The bench's multi-rank logic on CPU (gloo, world size 2): every rank runs its own
model, the timings reduce to the slowest rank, and the whole-job value counts the units
of all ranks (weak scaling, no collective on the data path)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_env() == (ws, rank, rank)
    mine = [10.0 + 5.0 * rank, 20.0 - 3.0 * rank]       # per-rank ms: rank 1 slower on the first
    mx = bench.reduce_max(mine, device="cpu")
    value = bench.whole_job_rate(1000, 4, ws, mx[0])
    dist.barrier()
    q.put((rank, mx, value))
    dist.destroy_process_group()


def test_two_rank_reduction_and_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, value in res:
        assert mx == [15.0, 20.0]                           # max over ranks, element-wise
        assert value == pytest.approx(2 * 1000 * 4 / 0.015)


def test_single_rank_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max([3.0, 4.0]) == [3.0, 4.0]
    assert bench.whole_job_rate(10, 2, 1, 1000.0) == pytest.approx(20.0)
