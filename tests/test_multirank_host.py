"""The multi-rank plumbing of bench.py (replicas, one lattice per rank) on
CPU: two gloo ranks in spawned processes, rendezvous on 127.0.0.1.  The job
time is the maximum over ranks and the whole-job value counts every rank's
site updates; no GPU is involved."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r "took" 1 + r seconds
    t = bench.max_over_ranks(1.0 + rank, dist, "cpu")
    out.put((rank, t, bench.dist_env(), bench.job_value(world, 1000, 10, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_job_time_is_the_max_over_two_gloo_ranks():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for rank, t, env, value in res:
        assert t == 2.0                              # the slowest rank sets the time
        assert env == (2, rank, rank)
        assert value == pytest.approx(2 * 1000 * 10 / 2.0 / 1e9)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_value(1, 10, 10, 1.0) == pytest.approx(1e-7)
