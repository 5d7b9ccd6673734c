"""The benchmark's multi-rank path on CPU ranks (gloo, world size 2): the
replicas share nothing on the data path; only the timing is combined (the
slowest rank's time) and the whole-job value is every rank's work over it.
The reference arm runs on rank 0 alone."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import sys
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    w, r, local = bench._dist()
    t = bench.reduce_max(1.5 + rank, w, torch.device("cpu"))
    v = bench.replica_value(1000.0, w, t)
    out.put((rank, w, r, local, t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, w, r, local, t, v in res:
        assert (w, r, local) == (2, rank, rank)
        assert t == 2.5                      # max of 1.5 and 2.5
        assert v == pytest.approx(2 * 1000.0 / 2.5)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import torch
    assert bench.reduce_max(3.0, 1, torch.device("cpu")) == 3.0
    assert bench.replica_value(10.0, 1, 2.0) == 5.0
