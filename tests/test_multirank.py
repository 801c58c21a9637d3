"""The multi-process path of the benchmark on CPU (gloo, world size 2): each
rank draws its own batch, and the job time is the maximum over ranks.  The
evaluation path has no collective (replicas / independent instances)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        w = bench.make_workload("batch", None, rank, B=6)
        mx = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 0.5])
        q.put((rank, [float(x) for x in w.inst.mass_msun], mx))
    finally:
        tdist.destroy_process_group()


def test_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict()
    for _ in range(2):
        r, masses, mx = q.get(timeout=120)
        res[r] = (masses, mx)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == res[1][1] == [2.0, 10.0, 0.5]
    assert len(res[0][0]) == len(res[1][0]) == 6
    assert res[0][0] != res[1][0]          # each rank its own parameter vectors


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 1.5]) == [3.0, 1.5]
