"""The multi-rank path of bench.py on CPU: two gloo ranks, as torchrun would start them.

Each rank runs an independent replica (distinct seed and Philox replica index, so distinct
thermal noise), the timed duration is the maximum over ranks, and the whole-job rate counts
the units of every rank.  No GPU is touched.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rep = bench.replica_of(rank, 2)
    local_ms = 100.0 + 50.0 * rank           # rank 1 is the slow one
    total = bench.max_over_ranks(local_ms, dist, "cpu")
    eta = oracle.normals(rep["seed"], rep["replica"], 0, 8, 0)
    gathered = [None] * world
    dist.all_gather_object(gathered, (rep, total, eta.tolist()))
    if rank == 0:
        out.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (rep0, t0, eta0), (rep1, t1, eta1) = res
    assert t0 == t1 == 150.0                                   # max over ranks, seen by every rank
    assert rep0 != rep1 and rep0["replica"] == 0 and rep1["replica"] == 1
    assert not np.array_equal(eta0, eta1)                      # independent noise per replica
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.whole_job_rate(2, 1000, 10, 150.0) == pytest.approx(2 * 1000 * 10 / 0.150)
